// walk.cu -- Sec. 4.2 step 3d, first half: one tree traversal per group
// builds the group's interaction list (Barnes' group walk): opened leaves
// become particle entries, accepted nodes become cell entries.  The walk is
// depth first in octant order, so both lists come out ordered by first
// particle.  A count pass sizes the lists, a fill pass writes them, and the
// particle entries are then expanded into the particle indices the force
// kernel reads.
//
// Opening test (integer boxes on the key grid, exact): per axis the gap in
// whole cells is delta = max(0, clo - ghi - 1, glo - chi - 1), d2 = sum of
// delta^2.  A node of level l (side 2^(21-l) cells) is opened iff
// fl(theta^2 * d2) < 4^(21-l), or d2 <= (r_coll * S)^2.  Both comparisons
// are monotone in the integer d2, so the host turns them into integer
// thresholds once per build: open iff d2 < D[l] or d2 <= RCQ.  With several
// patches a group walks the tree of its own patch (root = patch index), and
// RCQ is per patch (each patch has its own key grid).
#include <cmath>
#include <vector>

#include "bh_internal.cuh"

namespace bh {
namespace {

struct WalkParams {
    long long D[kLevels + 1];
    const long long* rcq;  // per patch
    const int64_t* off;    // patch particle offsets (np + 1)
    int np;
};

// Team walk: 8 lanes per group, 4 groups per warp.  A team evaluates a run of
// siblings (the children of one node, at most 8) at once, one node per lane,
// from one coalesced load of their records.  It emits, in order, the entries
// of the siblings before the first one that is opened and has children,
// keeps the rest of the run on its stack and descends into that one: the
// depth-first octant order of a one-thread walk, so both lists come out in
// order of first particle.
constexpr int kTeam = 8;
constexpr int kWalkThreads = 128;
constexpr int kTeamsPerBlock = kWalkThreads / kTeam;
constexpr int kStack = kLevels + 3;

template <bool FILL>
__global__ void __launch_bounds__(kWalkThreads) k_walk(int64_t ng, const int32_t* __restrict__ groups,
                                                      const WalkNode* __restrict__ wn,
                                                      const uint32_t* __restrict__ begin,
                                                      const uint32_t* __restrict__ end, WalkParams wp,
                                                      int64_t* __restrict__ np_io, int64_t* __restrict__ nc_io,
                                                      int64_t* __restrict__ nj_io, int32_t* __restrict__ P,
                                                      int32_t* __restrict__ C, unsigned long long* inter,
                                                      int64_t nn, int* status) {
    __shared__ int2 stk[kTeamsPerBlock][kStack];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int team = threadIdx.x / kTeam;  // team within the block
    const int tl = threadIdx.x & (kTeam - 1);
    const int tshift = lane & ~(kTeam - 1);  // the team's first lane in the warp
    const int64_t k = (int64_t)blockIdx.x * kTeamsPerBlock + team;
    const bool active = k < ng;
    int64_t np = 0, nc = 0, nj = 0, nown = 0, ni = 0, pbase = 0, cbase = 0;
    int glo0 = 0, glo1 = 0, glo2 = 0, ghi0 = 0, ghi1 = 0, ghi2 = 0;
    uint32_t gb = 0, ge = 0;
    long long rcq = 0;
    int sp = 0;
    if (active) {
        const int32_t g = groups[k];
        const WalkNode G = wn[g];
        gb = begin[g];
        ge = end[g];
        glo0 = (int)G.a.x; glo1 = (int)G.a.y; glo2 = (int)G.a.z;
        ghi0 = (int)G.b.x; ghi1 = (int)G.b.y; ghi2 = (int)G.b.z;
        ni = (int64_t)(ge - gb);
        if (FILL) {
            pbase = np_io[k];
            cbase = nc_io[k];
        }
        int root = 0;
        for (int lo = 0, hi = wp.np - 1; lo < hi;) {  // last patch starting at or before gb
            const int mid = (lo + hi + 1) >> 1;
            if (wp.off[mid] <= (int64_t)gb)
                lo = root = mid;
            else
                hi = mid - 1;
        }
        rcq = wp.rcq[root];
        if (tl == 0) stk[team][0] = make_int2(root, root + 1);
        sp = 1;
    }
    __syncwarp();
    while (__any_sync(FULL, sp > 0)) {
        const bool live = sp > 0;
        int s = 0, e = 0;
        if (live) {
            const int2 r = stk[team][sp - 1];
            s = r.x;
            e = r.y;
        }
        const int node = s + tl;
        bool has = live && node < e;
        if (has && (node < 0 || node >= nn)) {  // never taken for a valid tree
            atomicOr(status, kStatBounds);
            has = false;
        }
        int cls = -1;  // 0: accepted (cell entry), 1: opened leaf, 2: opened with children
        int nch = 0, fc = 0;
        uint32_t lb = 0, le = 0;
        if (has) {
            const WalkNode R = wn[node];
            const int lev = (int)(R.a.w & 0xffu);
            nch = (int)(R.a.w >> 8);
            fc = (int)R.b.w;
            const int d0 = max(0, max((int)R.a.x - ghi0 - 1, glo0 - (int)R.b.x - 1));
            const int d1 = max(0, max((int)R.a.y - ghi1 - 1, glo1 - (int)R.b.y - 1));
            const int d2i = max(0, max((int)R.a.z - ghi2 - 1, glo2 - (int)R.b.z - 1));
            const long long d2 = (long long)d0 * d0 + (long long)d1 * d1 + (long long)d2i * d2i;
            const bool open = d2 < wp.D[lev] || d2 <= rcq;
            cls = open ? (nch == 0 ? 1 : 2) : 0;
            if (cls == 1 && !FILL) {
                lb = begin[node];
                le = end[node];
            }
        }
        const unsigned b_int = (__ballot_sync(FULL, cls == 2) >> tshift) & 0xffu;
        const unsigned b_acc = (__ballot_sync(FULL, cls == 0) >> tshift) & 0xffu;
        const unsigned b_leaf = (__ballot_sync(FULL, cls == 1) >> tshift) & 0xffu;
        const int f = b_int ? __ffs(b_int) - 1 : kTeam;  // first sibling to descend into
        const unsigned below = (1u << f) - 1u;           // siblings whose entries go out now
        const unsigned emit_c = b_acc & below, emit_p = b_leaf & below;
        const unsigned lt = (1u << tl) - 1u;
        const bool my_c = (emit_c >> tl) & 1u, my_p = (emit_p >> tl) & 1u;
        if (FILL) {
            if (my_c) C[cbase + nc + __popc(emit_c & lt)] = node;
            if (my_p) P[pbase + np + __popc(emit_p & lt)] = node;
        } else if (my_p) {
            if (lb >= gb && lb < ge)
                nown += (int64_t)(le - lb);  // the group's own particles
            else
                nj += (int64_t)(le - lb);
        }
        nc += __popc(emit_c);
        np += __popc(emit_p);
        // children of the sibling descended into, from its lane
        const int src = tshift + (b_int ? f : tl);
        const int cfc = __shfl_sync(FULL, fc, src), cnch = __shfl_sync(FULL, nch, src);
        __syncwarp();
        if (live) {
            if (b_int) {
                if (s + f + 1 < e) {
                    if (tl == 0) stk[team][sp - 1] = make_int2(s + f + 1, e);
                } else {
                    --sp;
                }
                if (sp >= kStack || cfc < 0 || (int64_t)cfc + cnch > nn) {  // never taken for a valid tree
                    if (tl == 0) atomicOr(status, kStatBounds);
                    sp = 0;
                } else {
                    if (tl == 0) stk[team][sp] = make_int2(cfc, cfc + cnch);
                    ++sp;
                }
            } else {
                --sp;
            }
        }
        __syncwarp();
    }
    if (!FILL) {
        // own/other particle counts of the opened leaves: sum over the team
#pragma unroll
        for (int o = kTeam / 2; o > 0; o >>= 1) {
            nj += __shfl_xor_sync(FULL, nj, o);
            nown += __shfl_xor_sync(FULL, nown, o);
        }
        if (active && tl == 0) {
            np_io[k] = np;
            nc_io[k] = nc;
            nj_io[k] = nj;
        }
        // interaction counts: n_i * (list particles) and n_i * (list cells)
        unsigned long long ipp = 0, ipc = 0;
        if (active && tl == 0) {
            ipp = (unsigned long long)(ni * (nj + nown));
            ipc = (unsigned long long)(ni * nc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ipp += __shfl_xor_sync(FULL, ipp, o);
            ipc += __shfl_xor_sync(FULL, ipc, o);
        }
        if (lane == 0) {
            atomicAdd(&inter[0], ipp);
            atomicAdd(&inter[1], ipc);
        }
    }
}

// One warp per group: particle entries -> particle indices, leaving out the
// group's own particles (the force kernels evaluate those in a separate phase
// that excludes i = j).
__global__ void k_expand(int64_t ng, const int32_t* __restrict__ groups, const int64_t* __restrict__ pp_off,
                         const int32_t* __restrict__ P, const uint32_t* __restrict__ begin,
                         const uint32_t* __restrict__ end, const int64_t* __restrict__ jj_off,
                         uint32_t* __restrict__ JJ) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= ng) return;
    const int32_t g = groups[k];
    const uint32_t gb = begin[g], ge = end[g];
    const int64_t e0 = pp_off[k], e1 = pp_off[k + 1];
    int64_t jo = jj_off[k];
    for (int64_t e = e0; e < e1; e += 32) {
        uint32_t b = 0, cnt = 0;
        if (e + lane < e1) {
            const int32_t leaf = P[e + lane];
            b = begin[leaf];
            cnt = (b >= gb && b < ge) ? 0u : end[leaf] - b;
        }
        uint32_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, x, 31);
        const int64_t pos = jo + (x - cnt);
        for (uint32_t t = 0; t < cnt; ++t) JJ[pos + t] = b + t;
        jo += tot;
    }
}

__global__ void k_set_last(int64_t* off, int64_t ng, const unsigned long long* total) {
    off[ng] = (int64_t)*total;
}

WalkParams walk_params(const Ctx* c) {
    WalkParams w;
    const double th2 = c->prm.theta * c->prm.theta;
    const long long big = (long long)1 << 53;
    for (int l = 0; l <= kLevels; ++l) {
        const double s = std::ldexp(1.0, kLevels - l);
        const double s2 = s * s;
        if (th2 == 0.0) {
            w.D[l] = big;
            continue;
        }
        const double est = std::floor(s2 / th2);
        if (!(est < (double)big)) {
            w.D[l] = big;
            continue;
        }
        long long d = (long long)est;
        while (d > 0 && th2 * (double)(d - 1) >= s2) --d;
        while (!(th2 * (double)d >= s2)) ++d;
        w.D[l] = d;
    }
    w.rcq = c->d_rcq.p;
    w.off = c->d_off.p;
    w.np = c->n_patches;
    return w;
}

}  // namespace

int stage_lists(Ctx* c) {
    const int64_t ng = c->n_groups;
    BH_TRY(grow(c, c->cnt_p, (size_t)ng + 1, "list offsets P"));
    BH_TRY(grow(c, c->cnt_c, (size_t)ng + 1, "list offsets C"));
    BH_TRY(grow(c, c->cnt_j, (size_t)ng + 1, "list offsets J"));
    std::vector<long long> rcq(c->n_patches);
    for (int q = 0; q < c->n_patches; ++q) {
        const double r = c->prm.r_coll * c->h_box[8 * q + 4];
        const double r2 = r * r;
        rcq[q] = (r2 >= 9.0e18) ? (long long)9.0e18 : (long long)std::floor(r2);
    }
    BH_TRY(grow(c, c->d_rcq, rcq.size(), "walk contact thresholds"));
    BH_CUDA(c, cudaMemcpyAsync(c->d_rcq.p, rcq.data(), rcq.size() * sizeof(long long), cudaMemcpyHostToDevice,
                               c->stream));
    const WalkParams wp = walk_params(c);
    unsigned long long* inter = c->d_small + 8;
    BH_CUDA(c, cudaMemsetAsync(inter, 0, 2 * sizeof(unsigned long long), c->stream));
    const unsigned nb = blocks_for(ng, kTeamsPerBlock);
    k_walk<false><<<nb, kWalkThreads, 0, c->stream>>>(ng, c->groups.p, c->wnode.p, c->begin.p, c->end.p, wp, c->cnt_p.p,
                                             c->cnt_c.p, c->cnt_j.p, nullptr, nullptr, inter,
                                             c->n_nodes, c->d_status);
    BH_LAUNCH(c);
    DBuf<int64_t>* arr[3] = {&c->cnt_p, &c->cnt_c, &c->cnt_j};
    for (int a = 0; a < 3; ++a) {
        BH_TRY(scan_i64(c, arr[a]->p, arr[a]->p, ng, c->d_small + a));
        k_set_last<<<1, 1, 0, c->stream>>>(arr[a]->p, ng, c->d_small + a);
        BH_LAUNCH(c);
    }
    unsigned long long h[16];
    BH_CUDA(c, cudaMemcpyAsync(h, c->d_small, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    c->n_pp = (int64_t)h[0];
    c->n_pc = (int64_t)h[1];
    c->n_jj = (int64_t)h[2];
    c->n_int_pp = (int64_t)h[8];
    c->n_int_pc = (int64_t)h[9];
    BH_TRY(grow(c, c->P, (size_t)c->n_pp + 1, "particle lists"));
    BH_TRY(grow(c, c->C, (size_t)c->n_pc + 1, "cell lists"));
    BH_TRY(grow(c, c->JJ, (size_t)c->n_jj + 1, "list particle indices"));
    k_walk<true><<<nb, kWalkThreads, 0, c->stream>>>(ng, c->groups.p, c->wnode.p, c->begin.p, c->end.p, wp, c->cnt_p.p,
                                            c->cnt_c.p, c->cnt_j.p, c->P.p, c->C.p, inter,
                                            c->n_nodes, c->d_status);
    BH_LAUNCH(c);
    k_expand<<<blocks_for(ng * 32, 256), 256, 0, c->stream>>>(ng, c->groups.p, c->cnt_p.p, c->P.p, c->begin.p,
                                                             c->end.p, c->cnt_j.p, c->JJ.p);
    BH_LAUNCH(c);
    if (c->prm.precision == BH_PREC_FP32) BH_TRY(build_order32(c));
    return BH_OK;
}

}  // namespace bh
