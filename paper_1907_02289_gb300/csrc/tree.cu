// tree.cu -- Sec. 4.2 step 3a, second half, and the node refresh of the
// list-reusing step: level-by-level octree over sorted keys, integer node
// boxes on the key grid, node moments (mass, centre of mass, traceless
// quadrupole) and the groups (maximal nodes with at most n_g particles).
//
// Numbering: breadth first, key order within a level (a node's children are
// contiguous and in octant order).  A node at level l splits on the digit of
// level l+1 when it holds more than n_leaf particles and l < 21.
//
// Moments follow one fixed operation order (leaves: particles in order;
// internal nodes: children in octant order) with _rn intrinsics, so they do
// not depend on thread scheduling or on multiply-add contraction.
#include <algorithm>

#include "bh_internal.cuh"
#include "dfloat.cuh"

namespace bh {
namespace {

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x001f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x001f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x00000000001fffffull;
    return (uint32_t)x;
}

// Node range of one level: [ls, ls + cnt) as given, or from the device
// level bounds lvl[lev], lvl[lev + 1] (device-sized builds).
__device__ __forceinline__ void level_range(int64_t& ls, int64_t& cnt, const unsigned long long* lvl, int lev) {
    if (lvl) {
        ls = (int64_t)lvl[lev];
        cnt = (int64_t)lvl[lev + 1] - ls;
    }
}

// Roots: node q is the root of patch q (particles [off[q], off[q+1])).
__global__ void k_roots(uint8_t* level, uint32_t* begin, uint32_t* end, int32_t* parent,
                        const int64_t* __restrict__ off, int np) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    level[q] = 0;
    begin[q] = (uint32_t)off[q];
    end[q] = (uint32_t)off[q + 1];
    parent[q] = -1;
}

// Child boundaries of a node [b, e) of level lev: bnd[o] = first particle
// with octant digit >= o (o = 0..8), found by binary search; returns the
// number of non-empty children (0 when the node does not split).
__device__ __forceinline__ uint32_t split_bounds(const uint64_t* __restrict__ key, uint32_t b, uint32_t e, int lev,
                                                 int n_leaf, uint32_t (&bnd)[9]) {
    uint32_t nch = 0;
    if (e - b > (uint32_t)n_leaf && lev < kLevels) {
        const int shift = 3 * (kLevels - 1 - lev);
        uint32_t lo = b, prev = b;
        bnd[0] = b;
        for (int o = 1; o < 8; ++o) {
            uint32_t hi = e;
            while (lo < hi) {
                uint32_t mid = lo + ((hi - lo) >> 1);
                if ((int)((key[mid] >> shift) & 7u) < o)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            bnd[o] = lo;
            nch += (lo > prev);
            prev = lo;
        }
        bnd[8] = e;
        nch += (e > prev);
    }
    return nch;
}

// Child boundaries of each node of one level (9 per node, see split_bounds).
__global__ void k_split_count(const uint64_t* __restrict__ key, const uint32_t* __restrict__ begin,
                              const uint32_t* __restrict__ end, int64_t ls, int64_t cnt, int lev,
                              int n_leaf, uint32_t* __restrict__ nch_out, uint32_t* __restrict__ bnd) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    uint32_t bb[9];
    const uint32_t nch = split_bounds(key, begin[ls + t], end[ls + t], lev, n_leaf, bb);
    if (nch > 0)
#pragma unroll
        for (int o = 0; o < 9; ++o) bnd[9 * t + o] = bb[o];
    nch_out[t] = nch;
}

__global__ void k_split_write(const uint32_t* __restrict__ nch_in, const uint32_t* __restrict__ off,
                              const uint32_t* __restrict__ bnd, int64_t ls, int64_t cnt, int64_t le,
                              int lev, uint8_t* level, uint32_t* begin, uint32_t* end,
                              int32_t* parent, int32_t* first_child, uint8_t* nchild) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int64_t node = ls + t;
    const uint32_t nch = nch_in[t];
    if (nch == 0) {
        first_child[node] = -1;
        nchild[node] = 0;
        return;
    }
    const int64_t fc = le + off[t];
    first_child[node] = (int32_t)fc;
    nchild[node] = (uint8_t)nch;
    int k = 0;
    for (int o = 0; o < 8; ++o) {
        uint32_t b0 = bnd[9 * t + o], b1 = bnd[9 * t + o + 1];
        if (b1 > b0) {
            int64_t ch = fc + k++;
            level[ch] = (uint8_t)(lev + 1);
            begin[ch] = b0;
            end[ch] = b1;
            parent[ch] = (int32_t)node;
        }
    }
}

// ---- device-sized octree ---------------------------------------------------
// For a list-constructing step captured as one graph nothing is read back:
// the level bounds live on the device (sz[kSzLvl + l] = first node of level
// l), every level runs the same three launches (one node per thread, the
// threads striding over tiles of kLvTile nodes): counts and child bounds
// with per-tile sums; one block scanning the tile sums, which writes the next
// level's end, cut at the node capacity with the overflow flagged; the child
// writes.  The numbering is the one of the level loop above.
constexpr int kLvTile = 256;  // nodes per tile = threads per block

__global__ void k_lvl_init(unsigned long long* sz, int np) {
    if (threadIdx.x != 0) return;
    sz[kSzLvl] = 0;
    sz[kSzLvl + 1] = (unsigned long long)np;
    sz[kSzOvf] = 0;
    sz[kSzNeedNodes] = 0;
}

// Exclusive scan over the block (kLvTile threads); *total = block sum.
__device__ __forceinline__ uint32_t lv_exclusive(uint32_t v, uint32_t* wt, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = lane < kLvTile / 32 ? wt[lane] : 0u;
        uint32_t q = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, q, o);
            if (lane >= o) q += y;
        }
        if (lane < kLvTile / 32) wt[lane] = q - t;
        if (lane == kLvTile / 32 - 1) *total = q;
    }
    __syncthreads();
    const uint32_t r = wt[w] + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kLvTile) k_split_count_d(const uint64_t* __restrict__ key,
                                                           const uint32_t* __restrict__ begin,
                                                           const uint32_t* __restrict__ end,
                                                           const unsigned long long* __restrict__ sz, int lev,
                                                           int n_leaf, uint32_t* __restrict__ nch_out,
                                                           uint32_t* __restrict__ bnd, uint32_t* __restrict__ tsum) {
    __shared__ uint32_t wt[kLvTile / 32];
    __shared__ uint32_t tot;
    const int64_t ls = (int64_t)sz[kSzLvl + lev], cnt = (int64_t)sz[kSzLvl + lev + 1] - ls;
    const int64_t nt = (cnt + kLvTile - 1) / kLvTile;
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t t = tile * kLvTile + threadIdx.x;
        uint32_t nch = 0;
        if (t < cnt) {
            uint32_t bb[9];
            nch = split_bounds(key, begin[ls + t], end[ls + t], lev, n_leaf, bb);
            if (nch > 0)
#pragma unroll
                for (int o = 0; o < 9; ++o) bnd[9 * t + o] = bb[o];
            nch_out[t] = nch;
        }
        lv_exclusive(nch, wt, &tot);
        if (threadIdx.x == 0) tsum[tile] = tot;
    }
}

// One block: tile sums -> tile offsets; the next level ends at
// min(le + total, cap).
__global__ void __launch_bounds__(kLvTile) k_split_scan_d(unsigned long long* sz, int lev,
                                                          uint32_t* __restrict__ tsum, int64_t cap) {
    __shared__ uint32_t wt[kLvTile / 32];
    __shared__ uint32_t tot;
    const int64_t ls = (int64_t)sz[kSzLvl + lev], le = (int64_t)sz[kSzLvl + lev + 1], cnt = le - ls;
    const int64_t nt = (cnt + kLvTile - 1) / kLvTile;
    unsigned long long carry = 0;
    for (int64_t b0 = 0; b0 < nt; b0 += kLvTile) {
        const int64_t i = b0 + threadIdx.x;
        const uint32_t v = i < nt ? tsum[i] : 0u;
        const uint32_t e = lv_exclusive(v, wt, &tot);
        if (i < nt) tsum[i] = (uint32_t)(carry + e);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        const unsigned long long want = (unsigned long long)le + carry;
        sz[kSzLvl + lev + 2] = want < (unsigned long long)cap ? want : (unsigned long long)cap;
        if (want > (unsigned long long)cap) {
            sz[kSzOvf] |= kOvfNodes;
            if (want > sz[kSzNeedNodes]) sz[kSzNeedNodes] = want;
        }
    }
}

__global__ void __launch_bounds__(kLvTile) k_split_write_d(
    const unsigned long long* __restrict__ sz, int lev, const uint32_t* __restrict__ nch_in,
    const uint32_t* __restrict__ bnd, const uint32_t* __restrict__ tsum, int64_t cap, uint8_t* level,
    uint32_t* begin, uint32_t* end, int32_t* parent, int32_t* first_child, uint8_t* nchild) {
    __shared__ uint32_t wt[kLvTile / 32];
    __shared__ uint32_t tot;
    const int64_t ls = (int64_t)sz[kSzLvl + lev], le = (int64_t)sz[kSzLvl + lev + 1], cnt = le - ls;
    const int64_t nt = (cnt + kLvTile - 1) / kLvTile;
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t t = tile * kLvTile + threadIdx.x;
        const uint32_t nch = t < cnt ? nch_in[t] : 0u;
        const uint32_t off = tsum[tile] + lv_exclusive(nch, wt, &tot);
        if (t >= cnt) continue;
        const int64_t node = ls + t;
        if (nch == 0) {
            first_child[node] = -1;
            nchild[node] = 0;
            continue;
        }
        const int64_t fc = le + off;
        first_child[node] = (int32_t)fc;
        nchild[node] = (uint8_t)nch;
        int k = 0;
        for (int o = 0; o < 8; ++o) {
            const uint32_t b0 = bnd[9 * t + o], b1 = bnd[9 * t + o + 1];
            if (b1 > b0) {
                const int64_t ch = fc + k++;
                if (ch >= cap) continue;  // past the capacity (flagged by the scan)
                level[ch] = (uint8_t)(lev + 1);
                begin[ch] = b0;
                end[ch] = b1;
                parent[ch] = (int32_t)node;
            }
        }
    }
}

// Depth-first successor of node u's subtree: the node a pre-order walk
// visits after u when it does not descend into u.  Children of a node are
// consecutive ids, so that is u + 1 unless u is its parent's last child, in
// which case it is the parent's successor; a root has none (-1), which ends
// the walk of its patch.
__device__ __forceinline__ int32_t skip_of(int64_t u, const int32_t* __restrict__ parent,
                                           const int32_t* __restrict__ first_child,
                                           const uint8_t* __restrict__ nchild, int* status) {
    int64_t v = u;
    for (int up = 0; up <= kLevels + 1; ++up) {
        const int32_t p = parent[v];
        if (p < 0) return -1;
        if (v + 1 < (int64_t)first_child[p] + nchild[p]) return (int32_t)(v + 1);
        v = p;
    }
    atomicOr(status, kStatBounds);  // deeper than the key grid: never for a valid tree
    return -1;
}

// Integer tight boxes (grid coordinates recovered from the keys) and the
// packed records the walk reads (WalkNode).
__global__ void k_boxes(const uint64_t* __restrict__ key, int64_t ls, int64_t cnt,
                        const unsigned long long* __restrict__ lvl, int lev,
                        const uint8_t* __restrict__ level, const uint32_t* __restrict__ begin,
                        const uint32_t* __restrict__ end, const int32_t* __restrict__ parent,
                        const int32_t* __restrict__ first_child, const uint8_t* __restrict__ nchild,
                        uint32_t* qlo, uint32_t* qhi, WalkNode* wnode, int* status) {
    level_range(ls, cnt, lvl, lev);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = ls + t;
        uint32_t lo[3] = {kQMax, kQMax, kQMax}, hi[3] = {0, 0, 0};
        const int nc = nchild[k];
        if (nc == 0) {
            for (uint32_t i = begin[k]; i < end[k]; ++i) {
                uint64_t kk = key[i];
                uint32_t q[3] = {compact3(kk >> 2), compact3(kk >> 1), compact3(kk)};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    lo[a] = min(lo[a], q[a]);
                    hi[a] = max(hi[a], q[a]);
                }
            }
        } else {
            const int64_t f = first_child[k];
            for (int c = 0; c < nc; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    lo[a] = min(lo[a], qlo[3 * (f + c) + a]);
                    hi[a] = max(hi[a], qhi[3 * (f + c) + a]);
                }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            qlo[3 * k + a] = lo[a];
            qhi[3 * k + a] = hi[a];
        }
        WalkNode w;
        // a leaf carries its first particle and (up to kWalkCntMax - 1) its
        // particle count instead of a first child
        const uint32_t leafcnt = nc == 0 ? min(end[k] - begin[k], kWalkCntMax) : 0u;
        w.a = make_uint4(lo[0] | ((uint32_t)level[k] << kLevels) | (nc == 0 ? kWalkLeaf : 0u),
                         lo[1] | (leafcnt << kLevels), lo[2],
                         (uint32_t)skip_of(k, parent, first_child, nchild, status));
        w.b = make_uint4(hi[0], hi[1], hi[2], nc == 0 ? begin[k] : (uint32_t)first_child[k]);
        wnode[k] = w;
    }
}

// Moments of the nodes of one level (children already done).
template <int ORDER>
__global__ void k_moments(int64_t ls, int64_t cnt, const unsigned long long* __restrict__ lvl, int lev,
                          const uint32_t* __restrict__ begin,
                          const uint32_t* __restrict__ end, const int32_t* __restrict__ first_child,
                          const uint8_t* __restrict__ nchild, const double* __restrict__ x,
                          const double* __restrict__ y, const double* __restrict__ z,
                          const double* __restrict__ m, double* M, double* cx, double* cy,
                          double* cz, double* Q) {
    level_range(ls, cnt, lvl, lev);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = ls + t;
        const int nc = nchild[k];
        double Mk = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, c0, c1, c2;
        double q[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (nc == 0) {
            const uint32_t b = begin[k], e = end[k];
            for (uint32_t i = b; i < e; ++i) {
                const double mi = m[i];
                Mk = __dadd_rn(Mk, mi);
                sx = __dadd_rn(sx, __dmul_rn(mi, x[i]));
                sy = __dadd_rn(sy, __dmul_rn(mi, y[i]));
                sz = __dadd_rn(sz, __dmul_rn(mi, z[i]));
            }
            if (Mk > 0.0) {
                c0 = __ddiv_rn(sx, Mk);
                c1 = __ddiv_rn(sy, Mk);
                c2 = __ddiv_rn(sz, Mk);
            } else {
                c0 = x[b];
                c1 = y[b];
                c2 = z[b];
            }
            if (ORDER >= 2)
                for (uint32_t i = b; i < e; ++i) {
                    const double mi = m[i];
                    const double dx = __dsub_rn(x[i], c0), dy = __dsub_rn(y[i], c1), dz = __dsub_rn(z[i], c2);
                    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    const double tx = __dmul_rn(3.0, dx), ty = __dmul_rn(3.0, dy), tz = __dmul_rn(3.0, dz);
                    q[0] = __dadd_rn(q[0], __dmul_rn(mi, __dsub_rn(__dmul_rn(tx, dx), d2)));
                    q[1] = __dadd_rn(q[1], __dmul_rn(mi, __dsub_rn(__dmul_rn(ty, dy), d2)));
                    q[2] = __dadd_rn(q[2], __dmul_rn(mi, __dsub_rn(__dmul_rn(tz, dz), d2)));
                    q[3] = __dadd_rn(q[3], __dmul_rn(mi, __dmul_rn(tx, dy)));
                    q[4] = __dadd_rn(q[4], __dmul_rn(mi, __dmul_rn(tx, dz)));
                    q[5] = __dadd_rn(q[5], __dmul_rn(mi, __dmul_rn(ty, dz)));
                }
        } else {
            const int64_t f = first_child[k];
            for (int c = 0; c < nc; ++c) {
                const double Mc = M[f + c];
                Mk = __dadd_rn(Mk, Mc);
                sx = __dadd_rn(sx, __dmul_rn(Mc, cx[f + c]));
                sy = __dadd_rn(sy, __dmul_rn(Mc, cy[f + c]));
                sz = __dadd_rn(sz, __dmul_rn(Mc, cz[f + c]));
            }
            if (Mk > 0.0) {
                c0 = __ddiv_rn(sx, Mk);
                c1 = __ddiv_rn(sy, Mk);
                c2 = __ddiv_rn(sz, Mk);
            } else {
                c0 = cx[f];
                c1 = cy[f];
                c2 = cz[f];
            }
            if (ORDER >= 2)
                for (int c = 0; c < nc; ++c) {
                    const double Mc = M[f + c];
                    const double dx = __dsub_rn(cx[f + c], c0), dy = __dsub_rn(cy[f + c], c1),
                                 dz = __dsub_rn(cz[f + c], c2);
                    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    const double tx = __dmul_rn(3.0, dx), ty = __dmul_rn(3.0, dy), tz = __dmul_rn(3.0, dz);
                    const double* qc = Q + 6 * (f + c);
                    q[0] = __dadd_rn(__dadd_rn(q[0], qc[0]), __dmul_rn(Mc, __dsub_rn(__dmul_rn(tx, dx), d2)));
                    q[1] = __dadd_rn(__dadd_rn(q[1], qc[1]), __dmul_rn(Mc, __dsub_rn(__dmul_rn(ty, dy), d2)));
                    q[2] = __dadd_rn(__dadd_rn(q[2], qc[2]), __dmul_rn(Mc, __dsub_rn(__dmul_rn(tz, dz), d2)));
                    q[3] = __dadd_rn(__dadd_rn(q[3], qc[3]), __dmul_rn(Mc, __dmul_rn(tx, dy)));
                    q[4] = __dadd_rn(__dadd_rn(q[4], qc[4]), __dmul_rn(Mc, __dmul_rn(tx, dz)));
                    q[5] = __dadd_rn(__dadd_rn(q[5], qc[5]), __dmul_rn(Mc, __dmul_rn(ty, dz)));
                }
        }
        M[k] = Mk;
        cx[k] = c0;
        cy[k] = c1;
        cz[k] = c2;
#pragma unroll
        for (int a = 0; a < 6; ++a) Q[6 * k + a] = q[a];
    }
}

// Moments for the FP32 force path, all in FP32: offsets from a reference
// point inside the node (its first particle, or its first child's centre)
// are exact hi/lo differences; the centre of mass is kept as an FP32 hi/lo
// pair (reference + offset), mass and traceless quadrupole in FP32.
// Record layout: (c_hi, M), (c_lo, Qxx), (Qxy, Qxz, Qyy, Qyz).
__device__ __forceinline__ float dsub(float ah, float al, float bh, float bl) {
    return __fadd_rn(__fsub_rn(ah, bh), __fsub_rn(al, bl));
}

template <int ORDER>
__global__ void k_moments32(int64_t ls, int64_t cnt, const unsigned long long* __restrict__ lvl, int lev,
                            const uint32_t* __restrict__ begin,
                            const uint32_t* __restrict__ end, const int32_t* __restrict__ first_child,
                            const uint8_t* __restrict__ nchild, const float4* __restrict__ phi,
                            const float4* __restrict__ plo, float4* cell32, float* __restrict__ mlo) {
    level_range(ls, cnt, lvl, lev);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = ls + t;
        const int nc = nchild[k];
        float rh[3], rl[3];  // reference point (hi/lo)
        float Mk = 0.f, s[3] = {0.f, 0.f, 0.f}, q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // the mass also as a compensated sum of the (hi + lo) masses: the record
        // keeps Mk, mlo[k] the difference (for the refinement of the FP32 kernel)
        df Md = {0.f, 0.f};
        if (nc == 0) {
            const uint32_t b = begin[k], e = end[k];
            const float4 h0 = phi[b], l0 = plo[b];
            rh[0] = h0.x; rh[1] = h0.y; rh[2] = h0.z;
            rl[0] = l0.x; rl[1] = l0.y; rl[2] = l0.z;
            for (uint32_t i = b; i < e; ++i) {
                const float4 h = phi[i], l = plo[i];
                const float d[3] = {dsub(h.x, l.x, rh[0], rl[0]), dsub(h.y, l.y, rh[1], rl[1]), dsub(h.z, l.z, rh[2], rl[2])};
                Mk += h.w;
                Md = df_add(Md, {h.w, l.w});
#pragma unroll
                for (int a = 0; a < 3; ++a) s[a] = fmaf(h.w, d[a], s[a]);
            }
            const float inv = Mk > 0.f ? 1.f / Mk : 0.f;
            const float dc[3] = {s[0] * inv, s[1] * inv, s[2] * inv};
            if (ORDER >= 2)
                for (uint32_t i = b; i < e; ++i) {
                    const float4 h = phi[i], l = plo[i];
                    const float d[3] = {dsub(h.x, l.x, rh[0], rl[0]) - dc[0], dsub(h.y, l.y, rh[1], rl[1]) - dc[1],
                                        dsub(h.z, l.z, rh[2], rl[2]) - dc[2]};
                    const float d2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
                    const float m3 = 3.f * h.w;
                    q[0] = fmaf(h.w, fmaf(3.f * d[0], d[0], -d2), q[0]);
                    q[1] = fmaf(h.w, fmaf(3.f * d[1], d[1], -d2), q[1]);
                    q[2] = fmaf(h.w, fmaf(3.f * d[2], d[2], -d2), q[2]);
                    q[3] = fmaf(m3 * d[0], d[1], q[3]);
                    q[4] = fmaf(m3 * d[0], d[2], q[4]);
                    q[5] = fmaf(m3 * d[1], d[2], q[5]);
                }
#pragma unroll
            for (int a = 0; a < 3; ++a) s[a] = dc[a];
        } else {
            const int64_t f = first_child[k];
            const float4 c0h = cell32[3 * f], c0l = cell32[3 * f + 1];
            rh[0] = c0h.x; rh[1] = c0h.y; rh[2] = c0h.z;
            rl[0] = c0l.x; rl[1] = c0l.y; rl[2] = c0l.z;
            for (int cc = 0; cc < nc; ++cc) {
                const float4 h = cell32[3 * (f + cc)], l = cell32[3 * (f + cc) + 1];
                const float d[3] = {dsub(h.x, l.x, rh[0], rl[0]), dsub(h.y, l.y, rh[1], rl[1]), dsub(h.z, l.z, rh[2], rl[2])};
                Mk += h.w;
                Md = df_add(Md, {h.w, mlo[f + cc]});
#pragma unroll
                for (int a = 0; a < 3; ++a) s[a] = fmaf(h.w, d[a], s[a]);
            }
            const float inv = Mk > 0.f ? 1.f / Mk : 0.f;
            const float dc[3] = {s[0] * inv, s[1] * inv, s[2] * inv};
            if (ORDER >= 2)
                for (int cc = 0; cc < nc; ++cc) {
                    const float4 h = cell32[3 * (f + cc)], l = cell32[3 * (f + cc) + 1], u = cell32[3 * (f + cc) + 2];
                    const float D[3] = {dsub(h.x, l.x, rh[0], rl[0]) - dc[0], dsub(h.y, l.y, rh[1], rl[1]) - dc[1],
                                        dsub(h.z, l.z, rh[2], rl[2]) - dc[2]};
                    const float D2 = fmaf(D[0], D[0], fmaf(D[1], D[1], D[2] * D[2]));
                    const float Mc = h.w, m3 = 3.f * Mc;
                    q[0] += l.w + Mc * fmaf(3.f * D[0], D[0], -D2);
                    q[1] += u.z + Mc * fmaf(3.f * D[1], D[1], -D2);
                    q[2] += -(l.w + u.z) + Mc * fmaf(3.f * D[2], D[2], -D2);
                    q[3] += u.x + m3 * D[0] * D[1];
                    q[4] += u.y + m3 * D[0] * D[2];
                    q[5] += u.w + m3 * D[1] * D[2];
                }
#pragma unroll
            for (int a = 0; a < 3; ++a) s[a] = dc[a];
        }
        // centre = reference + offset, renormalised into a hi/lo pair
        float ch[3], cl[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = __fadd_rn(rl[a], s[a]);
            const float hi = __fadd_rn(rh[a], lo);
            ch[a] = hi;
            cl[a] = __fsub_rn(lo, __fsub_rn(hi, rh[a]));
        }
        mlo[k] = __fadd_rn(__fsub_rn(Md.hi, Mk), Md.lo);
        cell32[3 * k + 0] = make_float4(ch[0], ch[1], ch[2], Mk);
        cell32[3 * k + 1] = make_float4(cl[0], cl[1], cl[2], q[0]);
        cell32[3 * k + 2] = make_float4(q[3], q[4], q[1], q[5]);
    }
}

__global__ void k_group_mark(int64_t nn, const unsigned long long* __restrict__ dnn,
                             const uint32_t* __restrict__ begin, const uint32_t* __restrict__ end,
                             const int32_t* __restrict__ parent, const uint8_t* __restrict__ nchild,
                             int n_g, int32_t* __restrict__ gmark) {
    if (dnn) nn = min(nn, (int64_t)*dnn);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cnt = end[k] - begin[k];
        const bool small = cnt <= (uint32_t)n_g || nchild[k] == 0;
        // a root (of any patch: parent -1) or the child of a node above n_g
        const int32_t p = parent[k];
        const bool top = p < 0 || (end[p] - begin[p]) > (uint32_t)n_g;
        if (small && top) gmark[begin[k]] = (int32_t)k;
    }
}

__global__ void k_group_flag(const int32_t* __restrict__ gmark, int64_t n, uint32_t* __restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = gmark[i] >= 0 ? 1u : 0u;
}

__global__ void k_group_compact(const int32_t* __restrict__ gmark, const uint32_t* __restrict__ pos,
                                int64_t n, int32_t* __restrict__ groups) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && gmark[i] >= 0) groups[pos[i]] = gmark[i];
}

// Grid of a device-sized level launch: enough blocks for the previous
// build's nodes on that level with the build's room to grow (the kernels
// stride, so any count is covered; this only sets the parallelism).
unsigned dev_level_grid(const Ctx* c, int lev, int threads) {
    const auto& ls = c->lvl_start;
    const int64_t prev = lev + 1 < (int)ls.size() ? ls[lev + 1] - ls[lev] : 0;
    return blocks_for(prev + prev * c->tune.graph_room / 100 + 64, threads);
}

int grow_nodes(Ctx* c, size_t need) {
    if (need <= c->level.cap) return BH_OK;
    size_t cap = need + need / 2 + 1024;
    BH_TRY(grow(c, c->level, cap, "node level", true));
    BH_TRY(grow(c, c->nchild, cap, "node nchild", true));
    BH_TRY(grow(c, c->begin, cap, "node begin", true));
    BH_TRY(grow(c, c->end, cap, "node end", true));
    BH_TRY(grow(c, c->parent, cap, "node parent", true));
    BH_TRY(grow(c, c->first_child, cap, "node first_child", true));
    return BH_OK;
}

}  // namespace

// Device-sized octree: node arrays hold c->cap_nodes nodes (grown by the
// caller); c->n_nodes is that capacity until the sizes are read back.
int stage_octree_dev(Ctx* c) {
    const int np = c->n_patches;
    const int64_t cap = c->cap_nodes;
    const uint64_t* key = c->key[c->key_cur].p;
    const int64_t tiles = (cap + kLvTile - 1) / kLvTile;
    BH_TRY(grow(c, c->split_cnt, (size_t)cap, "split counts"));
    BH_TRY(grow(c, c->split_bnd, 9 * (size_t)cap, "split bounds"));
    BH_TRY(grow(c, c->split_off, (size_t)tiles + 1, "split tile sums"));
    k_roots<<<blocks_for(np, 64), 64, 0, c->stream>>>(c->level.p, c->begin.p, c->end.p, c->parent.p, c->d_off.p, np);
    BH_LAUNCH(c);
    k_lvl_init<<<1, 32, 0, c->stream>>>(c->d_sz, np);
    BH_LAUNCH(c);
    for (int lev = 0; lev <= kLevels; ++lev) {
        const unsigned grid = dev_level_grid(c, lev, kLvTile);
        k_split_count_d<<<grid, kLvTile, 0, c->stream>>>(key, c->begin.p, c->end.p, c->d_sz, lev, c->prm.n_leaf,
                                                         c->split_cnt.p, c->split_bnd.p, c->split_off.p);
        BH_LAUNCH(c);
        k_split_scan_d<<<1, kLvTile, 0, c->stream>>>(c->d_sz, lev, c->split_off.p, cap);
        BH_LAUNCH(c);
        k_split_write_d<<<grid, kLvTile, 0, c->stream>>>(c->d_sz, lev, c->split_cnt.p, c->split_bnd.p,
                                                         c->split_off.p, cap, c->level.p, c->begin.p, c->end.p,
                                                         c->parent.p, c->first_child.p, c->nchild.p);
        BH_LAUNCH(c);
    }
    c->n_nodes = cap;
    return BH_OK;
}

int stage_octree(Ctx* c) {
    if (c->dev_build) return stage_octree_dev(c);
    const int64_t n = c->n;
    const uint64_t* key = c->key[c->key_cur].p;
    const int np = c->n_patches;
    BH_TRY(grow_nodes(c, (size_t)(n / 2 + 64 + np)));
    k_roots<<<blocks_for(np, 64), 64, 0, c->stream>>>(c->level.p, c->begin.p, c->end.p, c->parent.p, c->d_off.p, np);
    BH_LAUNCH(c);
    c->lvl_start.assign({0, (int64_t)np});
    for (int lev = 0;; ++lev) {
        const int64_t ls = c->lvl_start[lev], le = c->lvl_start[lev + 1], cnt = le - ls;
        BH_TRY(grow(c, c->split_cnt, (size_t)cnt, "split counts"));
        BH_TRY(grow(c, c->split_off, (size_t)cnt, "split offsets"));
        BH_TRY(grow(c, c->split_bnd, (size_t)cnt * 9, "split bounds"));
        k_split_count<<<blocks_for(cnt, 128), 128, 0, c->stream>>>(key, c->begin.p, c->end.p, ls, cnt, lev,
                                                                   c->prm.n_leaf, c->split_cnt.p, c->split_bnd.p);
        BH_LAUNCH(c);
        BH_TRY(scan_u32(c, c->split_cnt.p, c->split_off.p, cnt, c->d_small));
        unsigned long long total = 0;
        BH_CUDA(c, cudaMemcpyAsync(&total, c->d_small, sizeof(total), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
        BH_TRY(grow_nodes(c, (size_t)(le + total)));
        k_split_write<<<blocks_for(cnt, 128), 128, 0, c->stream>>>(
            c->split_cnt.p, c->split_off.p, c->split_bnd.p, ls, cnt, le, lev, c->level.p, c->begin.p,
            c->end.p, c->parent.p, c->first_child.p, c->nchild.p);
        BH_LAUNCH(c);
        if (total == 0) break;
        c->lvl_start.push_back(le + (int64_t)total);
    }
    c->n_nodes = c->lvl_start.back();
    return BH_OK;
}

int stage_boxes(Ctx* c) {
    const int64_t nn = c->n_nodes;
    BH_TRY(grow(c, c->qlo, (size_t)nn * 3, "node qlo"));
    BH_TRY(grow(c, c->qhi, (size_t)nn * 3, "node qhi"));
    BH_TRY(grow(c, c->wnode, (size_t)nn, "walk records"));
    const unsigned long long* lvl = c->dev_build ? c->d_sz + kSzLvl : nullptr;
    const int depth = c->dev_build ? kLevels + 1 : (int)c->lvl_start.size() - 1;
    for (int lev = depth - 1; lev >= 0; --lev) {
        const int64_t ls = lvl ? 0 : c->lvl_start[lev], cnt = lvl ? 0 : c->lvl_start[lev + 1] - ls;
        k_boxes<<<lvl ? dev_level_grid(c, lev, 128) : blocks_for(cnt, 128), 128, 0, c->stream>>>(
            c->key[c->key_cur].p, ls, cnt, lvl, lev, c->level.p, c->begin.p, c->end.p, c->parent.p,
            c->first_child.p, c->nchild.p, c->qlo.p, c->qhi.p, c->wnode.p, c->d_status);
        BH_LAUNCH(c);
    }
    return BH_OK;
}

int stage_moments(Ctx* c, const bh_particles* p) {
    const int64_t nn = c->n_nodes;
    const bool f32 = c->prm.precision == BH_PREC_FP32;
    const unsigned long long* lvl = c->dev_build ? c->d_sz + kSzLvl : nullptr;
    const int depth = c->dev_build ? kLevels + 1 : (int)c->lvl_start.size() - 1;
    if (f32) {
        // FP32 path: hi/lo split of the particles, then FP32 moments with a
        // hi/lo centre (no FP64 arithmetic per node)
        BH_TRY(grow(c, c->cell32, (size_t)nn * 3, "FP32 cell records"));
        BH_TRY(grow(c, c->cell32lo, (size_t)nn, "FP32 cell mass corrections"));
        BH_TRY(stage_begin(c, BH_STAGE_SPLIT));
        BH_TRY(stage_split(c, p));
        BH_TRY(stage_end(c));
        BH_TRY(stage_begin(c, BH_STAGE_MOMENTS));
        for (int lev = depth - 1; lev >= 0; --lev) {
            const int64_t ls = lvl ? 0 : c->lvl_start[lev], cnt = lvl ? 0 : c->lvl_start[lev + 1] - ls;
            const unsigned nb = lvl ? dev_level_grid(c, lev, 128) : blocks_for(cnt, 128);
            if (c->prm.order >= 2)
                k_moments32<2><<<nb, 128, 0, c->stream>>>(ls, cnt, lvl, lev, c->begin.p, c->end.p, c->first_child.p,
                                                          c->nchild.p, c->phi.p, c->plo.p, c->cell32.p,
                                                          c->cell32lo.p);
            else
                k_moments32<1><<<nb, 128, 0, c->stream>>>(ls, cnt, lvl, lev, c->begin.p, c->end.p, c->first_child.p,
                                                          c->nchild.p, c->phi.p, c->plo.p, c->cell32.p,
                                                          c->cell32lo.p);
            BH_LAUNCH(c);
        }
        return stage_end(c);
    }
    return stage_moments64(c, p);
}

// FP64 node moments (the FP64 path's records; the FP32 path's potential
// diagnostic also uses them).
int stage_moments64(Ctx* c, const bh_particles* p) {
    const int64_t nn = c->n_nodes;
    const unsigned long long* lvl = c->dev_build ? c->d_sz + kSzLvl : nullptr;
    const int depth = c->dev_build ? kLevels + 1 : (int)c->lvl_start.size() - 1;
    BH_TRY(grow(c, c->M, (size_t)nn, "moments M"));
    BH_TRY(grow(c, c->cx, (size_t)nn, "moments cx"));
    BH_TRY(grow(c, c->cy, (size_t)nn, "moments cy"));
    BH_TRY(grow(c, c->cz, (size_t)nn, "moments cz"));
    BH_TRY(grow(c, c->Q, (size_t)nn * 6, "moments Q"));
    BH_TRY(stage_begin(c, BH_STAGE_MOMENTS));
    for (int lev = depth - 1; lev >= 0; --lev) {
        const int64_t ls = lvl ? 0 : c->lvl_start[lev], cnt = lvl ? 0 : c->lvl_start[lev + 1] - ls;
        const unsigned nb = lvl ? dev_level_grid(c, lev, 128) : blocks_for(cnt, 128);
#define BH_MOM(O)                                                                                              \
    k_moments<O><<<nb, 128, 0, c->stream>>>(ls, cnt, lvl, lev, c->begin.p, c->end.p, c->first_child.p, c->nchild.p, \
                                            p->x, p->y, p->z, p->m, c->M.p, c->cx.p, c->cy.p, c->cz.p, c->Q.p)
        if (c->prm.order >= 2)
            BH_MOM(2);
        else
            BH_MOM(1);
#undef BH_MOM
        BH_LAUNCH(c);
    }
    return stage_end(c);
}

int stage_groups(Ctx* c) {
    const int64_t n = c->n, nn = c->n_nodes;
    const bool dev = c->dev_build;
    BH_TRY(grow(c, c->gmark, (size_t)n, "group marks"));
    BH_TRY(grow(c, c->gflag, (size_t)n, "group flags"));
    BH_TRY(grow(c, c->gpos, (size_t)n, "group positions"));
    BH_CUDA(c, cudaMemsetAsync(c->gmark.p, 0xff, n * sizeof(int32_t), c->stream));
    k_group_mark<<<blocks_for(nn, 256), 256, 0, c->stream>>>(
        nn, dev ? c->d_sz + kSzLvl + kLevels + 2 : nullptr, c->begin.p, c->end.p, c->parent.p, c->nchild.p,
        c->prm.n_g, c->gmark.p);
    BH_LAUNCH(c);
    k_group_flag<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->gmark.p, n, c->gflag.p);
    BH_LAUNCH(c);
    unsigned long long* total = dev ? c->d_sz + kSzNg : c->d_small;
    BH_TRY(scan_u32(c, c->gflag.p, c->gpos.p, n, total));
    unsigned long long ng = (unsigned long long)n;  // device-sized: at most one group per particle
    if (!dev) {
        BH_CUDA(c, cudaMemcpyAsync(&ng, c->d_small, sizeof(ng), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    BH_TRY(grow(c, c->groups, (size_t)ng + 1, "groups"));
    k_group_compact<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->gmark.p, c->gpos.p, n, c->groups.p);
    BH_LAUNCH(c);
    c->n_groups = (int64_t)ng;
    return BH_OK;
}


}  // namespace bh
