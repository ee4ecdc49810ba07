// walk.cu -- Sec. 4.2 step 3d, first half: one tree traversal per group
// builds the group's interaction list (Barnes' group walk): opened leaves
// become particle entries, accepted nodes become cell entries.  The walk is
// depth first in octant order, so both lists come out ordered by first
// particle; it needs no stack, since every node carries the successor of its
// subtree.  A count pass sizes the lists and a fill pass writes them (16-byte
// stores); from the second build on, one pass both counts and writes each
// group's lists into a slot sized from the previous build, and a copy packs
// the slots (a group that outgrows its slot sends the build back to count
// and fill).  The particle entries are then expanded into the particle
// indices the force kernel reads.
//
// Opening test (integer boxes on the key grid, exact): per axis the gap in
// whole cells is delta = max(0, clo - ghi - 1, glo - chi - 1), d2 = sum of
// delta^2.  A node of level l (side 2^(21-l) cells) is opened iff
// fl(theta^2 * d2) < 4^(21-l), or d2 <= (r_coll * S)^2.  Both comparisons
// are monotone in the integer d2, so the host turns them into integer
// thresholds once per build: open iff d2 < D[l] or d2 <= RCQ.  With several
// patches a group walks the tree of its own patch (root = patch index), and
// RCQ is per patch (each patch has its own key grid).
//
// For the FP32 kernel the expansion puts a group's list particles in two
// runs: "near" leaves first, then "far" leaves, far meaning beyond contact
// reach with a margin (so no pair in them can touch) and a gap of at least an
// eighth of the group's largest side.  The kernel forms far separations from
// single FP32 coordinates relative to the group origin (the arithmetic of
// Sec. 4.7), whose error relative to the separation s is then at most about
// 2 u (1 + E / s) (E the group's extent from its centre, at most sqrt(3)
// times its side; u = 2^-24), i.e. 2 u (1 + 8 sqrt(3)) ~ 30 u, and skips the
// contact test for them.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bh_internal.cuh"

namespace bh {
namespace {

struct WalkParams {
    long long D[kLevels + 1];
    const long long* rcq;  // per patch
    const long long* rfar;    // per patch: d2 above this cannot hold a contact pair (margin included)
    const long long* period;  // per patch period of grid axis 0 (cylindrical frame), 0 = none
    const int64_t* off;    // patch particle offsets (np + 1)
    int np;
};

// Patch holding particle index gb: the last patch starting at or before it.
__device__ __forceinline__ int patch_of(const WalkParams& wp, uint32_t gb) {
    int root = 0;
    for (int lo = 0, hi = wp.np - 1; lo < hi;) {
        const int mid = (lo + hi + 1) >> 1;
        if (wp.off[mid] <= (int64_t)gb)
            lo = root = mid;
        else
            hi = mid - 1;
    }
    return root;
}

// Squared gap in whole cells between node box R and the group box [glo, ghi]
// (axis 0 periodic with the given period in cells when period > 0).
__device__ __forceinline__ long long box_gap2(const WalkNode& R, const int (&glo)[3], const int (&ghi)[3],
                                              int period) {
    const int lo0 = (int)(R.a.x & kQMax);
    const int t1 = lo0 - ghi[0] - 1, t2 = glo[0] - (int)R.b.x - 1;
    int d0 = max(0, max(t1, t2));
    if (period > 0 && d0 > 0)  // periodic phi axis: the shorter way round
        d0 = min(d0, max(0, t1 > 0 ? glo[0] + period - (int)R.b.x - 1 : lo0 + period - ghi[0] - 1));
    const int lo1 = (int)(R.a.y & kQMax);
    const int d1 = max(0, max(lo1 - ghi[1] - 1, glo[1] - (int)R.b.y - 1));
    const int d2 = max(0, max((int)R.a.z - ghi[2] - 1, glo[2] - (int)R.b.z - 1));
    return (long long)d0 * d0 + (long long)d1 * d1 + (long long)d2 * d2;
}

// Per-thread list writer: entries are gathered in registers and written as
// aligned 16-byte stores; the partial quads at the two ends of the thread's
// run [base, base + count) are written entry by entry, so no store touches
// another thread's run.  dst must be 16-byte aligned.
struct ListOut {
    int32_t* dst;
    int64_t base, pos, cap;  // entries at or past cap are counted, not written
    int32_t v0, v1, v2, v3;
    __device__ __forceinline__ int32_t at(int s) const { return s == 0 ? v0 : s == 1 ? v1 : s == 2 ? v2 : v3; }
    __device__ __forceinline__ void put_range(int64_t a, int64_t b) const {
        for (int64_t q = a; q < b; ++q) dst[q] = at((int)(q & 3));
    }
    __device__ __forceinline__ void put(int32_t v) {
        if (pos >= cap) {
            ++pos;
            return;
        }
        const int s = (int)(pos & 3);
        v0 = s == 0 ? v : v0;
        v1 = s == 1 ? v : v1;
        v2 = s == 2 ? v : v2;
        v3 = s == 3 ? v : v3;
        if (s == 3) {
            if (pos - 3 >= base)
                *reinterpret_cast<int4*>(dst + (pos - 3)) = make_int4(v0, v1, v2, v3);
            else
                put_range(base, pos + 1);
        }
        ++pos;
    }
    __device__ __forceinline__ void flush() const { put_range(max(base, min(pos, cap) & ~(int64_t)3), min(pos, cap)); }
};

// The walk is stackless: a node that is not descended into is followed by
// its subtree's successor (skip), an opened inner node by its first child,
// which visits the nodes in the same depth-first octant order as a stack.
// Modes: count (list sizes and interaction counts); fill (the lists, at the
// scanned offsets); stash (count, and write each group's lists into a slot
// of capP / capC entries at k * cap, flagging a group that does not fit).
// Count and stash also record the longest lists, which size the next
// build's slots.
constexpr int kWalkCount = 0, kWalkFill = 1, kWalkStash = 2;

template <int MODE>
__global__ void __launch_bounds__(128) k_walk(int64_t ng, const unsigned long long* __restrict__ dng,
                                              int64_t slots, const int32_t* __restrict__ groups,
                                              const WalkNode* __restrict__ wn,
                                              const uint32_t* __restrict__ begin,
                                              const uint32_t* __restrict__ end, WalkParams wp,
                                              int64_t* __restrict__ np_io, int64_t* __restrict__ nc_io,
                                              int64_t* __restrict__ nj_io, int32_t* __restrict__ P,
                                              int32_t* __restrict__ C, unsigned long long* inter,
                                              int64_t nn, int* status, int64_t capP, int64_t capC,
                                              unsigned long long* longest, unsigned long long* overflow) {
    constexpr bool WRITE = MODE != kWalkCount, COUNT = MODE != kWalkFill;
    if (dng) ng = min(ng, (int64_t)*dng);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ng; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = base + threadIdx.x;
        bool active = k < ng;
        if (MODE == kWalkFill && active && slots >= 0)  // only the groups that did not fit their slot
            active = !(k < slots && np_io[k + 1] - np_io[k] <= capP && nc_io[k + 1] - nc_io[k] <= capC);
        int64_t np = 0, nc = 0, nj = 0, ni = 0, nown = 0;
        if (active) {
            const int32_t g = groups[k];
            const WalkNode G = wn[g];
            const uint32_t gb = begin[g], ge = end[g];
            const int glo[3] = {(int)(G.a.x & kQMax), (int)(G.a.y & kQMax), (int)G.a.z};
            const int ghi[3] = {(int)G.b.x, (int)G.b.y, (int)G.b.z};
            ni = (int64_t)(end[g] - begin[g]);
            ListOut po{P, 0, 0, INT64_MAX, 0, 0, 0, 0}, co{C, 0, 0, INT64_MAX, 0, 0, 0, 0};
            if (MODE == kWalkFill) {
                po.base = po.pos = np_io[k];
                co.base = co.pos = nc_io[k];
            } else if (MODE == kWalkStash && (slots < 0 || k < slots)) {
                po.dst = P + k * capP;
                po.cap = capP;
                co.dst = C + k * capC;
                co.cap = capC;
            } else if (MODE == kWalkStash) {  // no slot: counted only, filled later
                po.cap = 0;
                co.cap = 0;
            }
            const int root = patch_of(wp, gb);
            const long long rcq = wp.rcq[root];
            const int period = (int)wp.period[root];
            int node = root;
            for (int64_t visits = 0;; ++visits) {
                const WalkNode R = wn[node];
                const int after = (int)R.a.w;
                const int lev = (int)((R.a.x >> kLevels) & 31u);
                const bool leaf = (R.a.x & kWalkLeaf) != 0;
                const long long d2 = box_gap2(R, glo, ghi, period);
                const bool open = d2 < wp.D[lev] || d2 <= rcq;
                int next = after;
                if (open) {
                    if (leaf) {
                        if (WRITE) po.put(node);
                        ++np;
                        const uint32_t lb = R.b.w;
                        uint32_t lc = R.a.y >> kLevels;
                        if (lc == kWalkCntMax) lc = end[node] - lb;
                        if (lb >= gb && lb < ge)
                            nown += (int64_t)lc;  // the group's own particles
                        else
                            nj += (int64_t)lc;
                    } else {
                        next = (int)R.b.w;
                    }
                } else {
                    if (WRITE) co.put(node);
                    ++nc;
                }
                if (next < 0) break;
                if (next >= nn || visits >= nn) {  // never taken for a valid tree
                    atomicOr(status, kStatBounds);
                    break;
                }
                node = next;
            }
            if (WRITE) {
                po.flush();
                co.flush();
            }
            if (MODE == kWalkStash && (np > po.cap || nc > co.cap)) atomicOr(overflow, 1ull);
            if (COUNT) {
                np_io[k] = np;
                nc_io[k] = nc;
                nj_io[k] = nj;
            }
        }
        if (COUNT) {
            // interaction counts: n_i * (list particles) and n_i * (list cells);
            // longest particle and cell lists
            unsigned long long ipp = (unsigned long long)(ni * (nj + nown)), ipc = (unsigned long long)(ni * nc);
            unsigned long long lp = (unsigned long long)np, lc = (unsigned long long)nc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ipp += __shfl_xor_sync(0xffffffffu, ipp, o);
                ipc += __shfl_xor_sync(0xffffffffu, ipc, o);
                lp = max(lp, __shfl_xor_sync(0xffffffffu, lp, o));
                lc = max(lc, __shfl_xor_sync(0xffffffffu, lc, o));
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&inter[0], ipp);
                atomicAdd(&inter[1], ipc);
                atomicMax(&longest[0], lp);
                atomicMax(&longest[1], lc);
            }
        }
    }
}

// One warp per group: particle entries -> particle indices, leaving out the
// group's own particles (the force kernels evaluate those in a separate phase
// that excludes i = j).  SPLIT: near leaves first, far leaves after them
// (each run in list order); jm[k] = index of the first far particle, and
// the far interactions n_i x (far particles) are summed into *n_far.
template <bool SPLIT>
__global__ void k_expand(int64_t ng, const unsigned long long* __restrict__ dng, const int32_t* __restrict__ groups,
                         const int64_t* __restrict__ pp_off, const int32_t* __restrict__ P, const uint32_t* __restrict__ begin,
                         const uint32_t* __restrict__ end, const WalkNode* __restrict__ wn, WalkParams wp,
                         const int64_t* __restrict__ jj_off, uint32_t* __restrict__ JJ, int64_t* __restrict__ jm,
                         unsigned long long* n_far) {
    if (dng) ng = min(ng, (int64_t)*dng);
    const int lane = threadIdx.x & 31;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < ng; k += wstride) {
        const int32_t g = groups[k];
        const uint32_t gb = begin[g], ge = end[g];
        const int64_t e0 = pp_off[k], e1 = pp_off[k + 1];
        int glo[3] = {0, 0, 0}, ghi[3] = {0, 0, 0};
        long long rfar = 0, ext2 = 0;
        int period = 0;
        if (SPLIT) {
            const WalkNode G = wn[g];
            glo[0] = (int)(G.a.x & kQMax); glo[1] = (int)(G.a.y & kQMax); glo[2] = (int)G.a.z;
            ghi[0] = (int)G.b.x; ghi[1] = (int)G.b.y; ghi[2] = (int)G.b.z;
            const long long ext = max(ghi[0] - glo[0], max(ghi[1] - glo[1], ghi[2] - glo[2])) + 1;
            ext2 = ext * ext;
            const int root = patch_of(wp, gb);
            rfar = wp.rfar[root];
            period = (int)wp.period[root];
        }
        // leaf entry e -> (first particle, count; 0 for the group's own
        // leaves) from its walk record, and whether it is far
        auto entry = [&](int64_t e, uint32_t& b, uint32_t& cnt, bool& far) {
            b = 0;
            cnt = 0;
            far = false;
            if (e < e1) {
                const int32_t leaf = P[e];
                const WalkNode R = wn[leaf];
                b = R.b.w;
                cnt = R.a.y >> kLevels;
                if (cnt == kWalkCntMax) cnt = end[leaf] - b;
                if (b >= gb && b < ge) cnt = 0;
                if (SPLIT && cnt > 0) {
                    const long long d2 = box_gap2(R, glo, ghi, period);
                    far = d2 > rfar && 64 * d2 >= ext2;
                }
            }
        };
        int64_t jn = jj_off[k], jf = jn;
        if (SPLIT) {  // far run starts after every near particle
            uint32_t near = 0;
            for (int64_t e = e0 + lane; e < e1; e += 32) {
                uint32_t b, cnt;
                bool far;
                entry(e, b, cnt, far);
                near += far ? 0u : cnt;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) near += __shfl_xor_sync(0xffffffffu, near, o);
            jf = jn + near;
            if (lane == 0) {
                jm[k] = jf;
                const unsigned long long ni = ge - gb;
                atomicAdd(n_far, ni * (unsigned long long)(jj_off[k + 1] - jf));
            }
        }
        for (int64_t e = e0; e < e1; e += 32) {
            uint32_t b, cnt;
            bool far;
            entry(e + lane, b, cnt, far);
            const uint32_t cn = far ? 0u : cnt, cf = far ? cnt : 0u;
            uint32_t xn = cn, xf = cf;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t yn = __shfl_up_sync(0xffffffffu, xn, o);
                const uint32_t yf = __shfl_up_sync(0xffffffffu, xf, o);
                if (lane >= o) {
                    xn += yn;
                    xf += yf;
                }
            }
            const uint32_t tn = __shfl_sync(0xffffffffu, xn, 31), tf = __shfl_sync(0xffffffffu, xf, 31);
            const int64_t pos = far ? jf + (xf - cf) : jn + (xn - cn);
            for (uint32_t t = 0; t < cnt; ++t) JJ[pos + t] = b + t;
            jn += tn;
            jf += tf;
        }
    }
}

// One warp per group: the group's stashed lists (slots of capP / capC
// entries) to their places in the packed lists.  slots >= 0 (device-sized
// build): only the groups below slots whose lists fit their slot.
__global__ void k_unstash(int64_t ng, const unsigned long long* __restrict__ dng, int64_t slots,
                          const int64_t* __restrict__ pp_off, const int64_t* __restrict__ pc_off,
                          const int32_t* __restrict__ sP, const int32_t* __restrict__ sC, int64_t capP,
                          int64_t capC, int32_t* __restrict__ P, int32_t* __restrict__ C) {
    if (dng) ng = min(ng, (int64_t)*dng);
    const int lane = threadIdx.x & 31;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < ng; k += wstride) {
        const int64_t p0 = pp_off[k], np = pp_off[k + 1] - p0, c0 = pc_off[k], nc = pc_off[k + 1] - c0;
        if (slots >= 0 && !(k < slots && np <= capP && nc <= capC)) continue;
        // four loads in flight per lane
        auto copy = [&](int32_t* __restrict__ dst, const int32_t* __restrict__ src, int64_t cnt) {
            for (int64_t t0 = 0; t0 < cnt; t0 += 128) {
                int32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t t = t0 + 32 * u + lane;
                    v[u] = t < cnt ? src[t] : 0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t t = t0 + 32 * u + lane;
                    if (t < cnt) dst[t] = v[u];
                }
            }
        };
        copy(P + p0, sP + k * capP, np);
        copy(C + c0, sC + k * capC, nc);
    }
}

__global__ void k_set_last(int64_t* off, int64_t ng, const unsigned long long* dng, const unsigned long long* total) {
    off[dng ? min(ng, (int64_t)*dng) : ng] = (int64_t)*total;
}

// Walk thresholds per patch from its key grid (S = 2^21 / L).  Contact
// reach in grid units: Cartesian r_coll S; cylindrical (phi, r, z): two
// particles within r_coll have |dr|, |dz| <= r_coll and a phi difference of
// at most ~r_coll / r_min, so (r_coll / r_min + 4e-6) S bounds their grid
// distance (4e-6 covers twice the FP32 tree coordinates' error), and the phi
// axis wraps after floor(2 pi S) cells.  rcq = floor(reach^2); the far threshold
// of the split expansion widens the reach by 1e-5 of itself plus two cells,
// so that no rounding of a coordinate into its cell can put a touching pair
// into a far leaf.  Round-to-nearest operations throughout (no contraction).
__global__ void k_walk_thresholds(const double* __restrict__ box, int np, double r_coll, int cyl,
                                  long long* __restrict__ rcq, long long* __restrict__ rfar,
                                  long long* __restrict__ period) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    const double S = __ddiv_rn(2097152.0, box[8 * q + 3]);
    double a;
    long long per = 0;
    if (cyl) {
        a = __ddiv_rn(r_coll, box[8 * q + 1]);
        a = __dadd_rn(a, 4e-6);
        a = __dmul_rn(a, S);
        per = (long long)floor(__dmul_rn(6.283185307179586, S));
    } else {
        a = __dmul_rn(r_coll, S);
    }
    const double r2 = __dmul_rn(a, a);
    rcq[q] = (r2 >= 9.0e18) ? (long long)9.0e18 : (long long)floor(r2);
    const double w = r_coll > 0.0 ? __dadd_rn(__dmul_rn(a, 1.0 + 1e-5), 2.0) : 0.0;
    const double w2 = __dmul_rn(w, w);
    rfar[q] = (w2 >= 9.0e18) ? (long long)9.0e18 : (long long)floor(w2);
    period[q] = per;
}

// Device-sized build: the list totals against the buffers' room.
__global__ void k_list_room(const unsigned long long* __restrict__ tot, long long roomP, long long roomC,
                            long long roomJ, unsigned long long* sz) {
    if (threadIdx.x != 0) return;
    if ((long long)tot[0] > roomP || (long long)tot[1] > roomC || (long long)tot[2] > roomJ) sz[kSzOvf] |= kOvfLists;
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
    w.rfar = c->d_rfar.p;
    w.period = c->d_period.p;
    w.off = c->d_off.p;
    w.np = c->n_patches;
    return w;
}

}  // namespace

namespace {

// Walk thresholds of every patch, on the device from the root boxes.
int walk_thresholds(Ctx* c) {
    const int np = c->n_patches;
    BH_TRY(grow(c, c->d_rcq, (size_t)np, "walk contact thresholds"));
    BH_TRY(grow(c, c->d_rfar, (size_t)np, "far thresholds"));
    BH_TRY(grow(c, c->d_period, (size_t)np, "walk periods"));
    k_walk_thresholds<<<blocks_for(np, 64), 64, 0, c->stream>>>(c->d_box, np, c->prm.r_coll, c->prm.key_frame == 1,
                                                                c->d_rcq.p, c->d_rfar.p, c->d_period.p);
    BH_LAUNCH(c);
    return BH_OK;
}

// Particle entries -> particle indices (near run, then far run for the FP32
// kernel) and the FP32 kernel's group order.
int expand_lists(Ctx* c, const WalkParams& wp, const unsigned long long* dng, unsigned grid) {
    const int64_t ng = c->n_groups;
    const bool split = c->prm.precision == BH_PREC_FP32;
    unsigned long long* n_far = c->d_small + 10;
    if (split) {
        BH_TRY(grow(c, c->cnt_jm, (size_t)ng + 1, "list split points"));
        BH_CUDA(c, cudaMemsetAsync(n_far, 0, sizeof(unsigned long long), c->stream));
    }
    auto expand = split ? k_expand<true> : k_expand<false>;
    expand<<<grid, 256, 0, c->stream>>>(ng, dng, c->groups.p, c->cnt_p.p, c->P.p, c->begin.p, c->end.p, c->wnode.p,
                                        wp, c->cnt_j.p, c->JJ.p, split ? c->cnt_jm.p : nullptr, n_far);
    BH_LAUNCH(c);
    return BH_OK;
}

}  // namespace

int stage_lists(Ctx* c) {
    const int64_t ng = c->n_groups;
    BH_TRY(grow(c, c->cnt_p, (size_t)ng + 1, "list offsets P"));
    BH_TRY(grow(c, c->cnt_c, (size_t)ng + 1, "list offsets C"));
    BH_TRY(grow(c, c->cnt_j, (size_t)ng + 1, "list offsets J"));
    BH_TRY(walk_thresholds(c));
    const WalkParams wp = walk_params(c);
    unsigned long long* inter = c->d_small + 8;
    unsigned long long* overflow = c->d_small + 11;
    unsigned long long* longest = c->d_small + 12;  // two words
    // One walk when the previous build gave slot sizes and the slots take
    // at most 4x the previous lists' storage; else (and after an overflow)
    // a count walk and a fill walk.
    const int64_t capP = c->walk_cap_p, capC = c->walk_cap_c;
    // (a list capacity bounds the entries held, so it rules out the slots)
    bool stash = capP > 0 && capC > 0 && c->prm.list_capacity == 0 &&
                 (double)ng * (double)(capP + capC) <= 4.0 * (double)(c->n_pp + c->n_pc) + 1.0e6;
    if (stash) {
        BH_TRY(grow(c, c->stash_p, (size_t)(ng * capP), "stashed particle lists"));
        BH_TRY(grow(c, c->stash_c, (size_t)(ng * capC), "stashed cell lists"));
    }
    BH_CUDA(c, cudaMemsetAsync(inter, 0, 6 * sizeof(unsigned long long), c->stream));  // words 8..13
    const unsigned nb = blocks_for(ng, 128);
    if (stash)
        k_walk<kWalkStash><<<nb, 128, 0, c->stream>>>(
            ng, nullptr, -1, c->groups.p, c->wnode.p, c->begin.p, c->end.p, wp, c->cnt_p.p, c->cnt_c.p,
            c->cnt_j.p, c->stash_p.p, c->stash_c.p, inter, c->n_nodes, c->d_status, capP, capC, longest, overflow);
    else
        k_walk<kWalkCount><<<nb, 128, 0, c->stream>>>(
            ng, nullptr, -1, c->groups.p, c->wnode.p, c->begin.p, c->end.p, wp, c->cnt_p.p, c->cnt_c.p,
            c->cnt_j.p, nullptr, nullptr, inter, c->n_nodes, c->d_status, 0, 0, longest, overflow);
    BH_LAUNCH(c);
    DBuf<int64_t>* arr[3] = {&c->cnt_p, &c->cnt_c, &c->cnt_j};
    for (int a = 0; a < 3; ++a) {
        BH_TRY(scan_i64(c, arr[a]->p, arr[a]->p, ng, c->d_small + a));
        k_set_last<<<1, 1, 0, c->stream>>>(arr[a]->p, ng, nullptr, c->d_small + a);
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
    c->list_overflowed = false;
    if (c->prm.list_capacity > 0 && c->n_pp + c->n_pc + c->n_jj > c->prm.list_capacity) {
        c->list_overflowed = true;
        c->need_pp = c->n_pp;
        c->need_pc = c->n_pc;
        c->need_jj = c->n_jj;
        return fail(c, BH_E_LIST_OVERFLOW,
                    "the lists need %lld entries (%lld leaf, %lld cell, %lld list-particle), list_capacity is %lld",
                    (long long)(c->n_pp + c->n_pc + c->n_jj), (long long)c->n_pp, (long long)c->n_pc,
                    (long long)c->n_jj, (long long)c->prm.list_capacity);
    }
    BH_TRY(grow(c, c->P, (size_t)c->n_pp + 1, "particle lists"));
    BH_TRY(grow(c, c->C, (size_t)c->n_pc + 1, "cell lists"));
    BH_TRY(grow(c, c->JJ, (size_t)c->n_jj + 1, "list particle indices"));
    if (stash && h[11] == 0) {
        k_unstash<<<blocks_for(ng * 32, 256), 256, 0, c->stream>>>(ng, nullptr, -1, c->cnt_p.p, c->cnt_c.p,
                                                                   c->stash_p.p, c->stash_c.p, capP, capC, c->P.p,
                                                                   c->C.p);
        ++c->n_one_walk_builds;
    } else {
        k_walk<kWalkFill><<<nb, 128, 0, c->stream>>>(
            ng, nullptr, -1, c->groups.p, c->wnode.p, c->begin.p, c->end.p, wp, c->cnt_p.p, c->cnt_c.p,
            c->cnt_j.p, c->P.p, c->C.p, inter, c->n_nodes, c->d_status, 0, 0, longest, overflow);
    }
    BH_LAUNCH(c);
    // slots of the next build: the longest lists of this one plus a quarter,
    // in whole 16-byte units
    c->walk_cap_p = (int64_t)(((h[12] + h[12] / 4 + 4) + 3) & ~3ull);
    c->walk_cap_c = (int64_t)(((h[13] + h[13] / 4 + 4) + 3) & ~3ull);
    BH_TRY(expand_lists(c, wp, nullptr, blocks_for(ng * 32, 256)));
    c->n_int_pp_far = 0;
    if (c->prm.precision == BH_PREC_FP32) {
        unsigned long long hf = 0;
        BH_CUDA(c, cudaMemcpyAsync(&hf, c->d_small + 10, sizeof(hf), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
        c->n_int_pp_far = (int64_t)hf;
        BH_TRY(build_order32(c));
    }
    return BH_OK;
}

// Device-sized list build, first part: the walk of every group (counting,
// and writing each group's lists into its slot when it has one that fits:
// c->dev_slots slots of walk_cap_p / walk_cap_c entries), the list offsets,
// and the room check of the totals against the P, C and JJ buffers as they
// are (kOvfLists).  Group count on the device; c->n_groups is its bound.
int stage_lists_dev_walk(Ctx* c) {
    const int64_t ng = c->n_groups;
    const unsigned long long* dng = c->d_sz + kSzNg;
    BH_TRY(grow(c, c->cnt_p, (size_t)ng + 1, "list offsets P"));
    BH_TRY(grow(c, c->cnt_c, (size_t)ng + 1, "list offsets C"));
    BH_TRY(grow(c, c->cnt_j, (size_t)ng + 1, "list offsets J"));
    BH_TRY(walk_thresholds(c));
    const WalkParams wp = walk_params(c);
    unsigned long long* inter = c->d_small + 8;
    unsigned long long* overflow = c->d_small + 11;
    unsigned long long* longest = c->d_small + 12;
    const int64_t slots = c->dev_slots, capP = c->walk_cap_p, capC = c->walk_cap_c;
    BH_TRY(grow(c, c->stash_p, (size_t)std::max<int64_t>(1, slots * capP), "stashed particle lists"));
    BH_TRY(grow(c, c->stash_c, (size_t)std::max<int64_t>(1, slots * capC), "stashed cell lists"));
    BH_CUDA(c, cudaMemsetAsync(inter, 0, 6 * sizeof(unsigned long long), c->stream));  // words 8..13
    const unsigned nb = blocks_for(std::max<int64_t>(slots, 1), 128);
    k_walk<kWalkStash><<<nb, 128, 0, c->stream>>>(ng, dng, slots, c->groups.p, c->wnode.p, c->begin.p,
                                                  c->end.p, wp, c->cnt_p.p, c->cnt_c.p, c->cnt_j.p, c->stash_p.p,
                                                  c->stash_c.p, inter, c->n_nodes, c->d_status, capP, capC, longest,
                                                  overflow);
    BH_LAUNCH(c);
    DBuf<int64_t>* arr[3] = {&c->cnt_p, &c->cnt_c, &c->cnt_j};
    for (int a = 0; a < 3; ++a) {
        BH_TRY(scan_i64(c, arr[a]->p, arr[a]->p, ng, c->d_small + a, dng));
        k_set_last<<<1, 1, 0, c->stream>>>(arr[a]->p, ng, dng, c->d_small + a);
        BH_LAUNCH(c);
    }
    k_list_room<<<1, 32, 0, c->stream>>>(c->d_small, (long long)c->P.cap - 1, (long long)c->C.cap - 1,
                                         (long long)c->JJ.cap - 1, c->d_sz);
    BH_LAUNCH(c);
    return BH_OK;
}

// Second part (issued to run only when the lists fit): the groups' lists
// from their slots or, for the groups without a fitting slot, from a second
// walk; the expansion into particle indices; the FP32 kernel's group order.
int stage_lists_dev_fill(Ctx* c) {
    const int64_t ng = c->n_groups;
    const unsigned long long* dng = c->d_sz + kSzNg;
    const WalkParams wp = walk_params(c);
    const int64_t slots = c->dev_slots, capP = c->walk_cap_p, capC = c->walk_cap_c;
    const unsigned grid = blocks_for(std::max<int64_t>(slots, 1) * 32, 256);  // a warp per expected group
    k_unstash<<<grid, 256, 0, c->stream>>>(ng, dng, slots, c->cnt_p.p, c->cnt_c.p, c->stash_p.p, c->stash_c.p, capP,
                                           capC, c->P.p, c->C.p);
    BH_LAUNCH(c);
    k_walk<kWalkFill><<<blocks_for(std::max<int64_t>(slots, 1), 128), 128, 0, c->stream>>>(
        ng, dng, slots, c->groups.p, c->wnode.p, c->begin.p, c->end.p, wp, c->cnt_p.p, c->cnt_c.p,
        c->cnt_j.p, c->P.p, c->C.p, c->d_small + 8, c->n_nodes, c->d_status, capP, capC, c->d_small + 12,
        c->d_small + 11);
    BH_LAUNCH(c);
    BH_TRY(expand_lists(c, wp, dng, grid));
    if (c->prm.precision == BH_PREC_FP32) BH_TRY(build_order32(c));
    return BH_OK;
}

}  // namespace bh
