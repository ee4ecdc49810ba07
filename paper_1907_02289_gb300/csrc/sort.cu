// sort.cu -- Sec. 4.2 step 3a, first half: root box, Morton keys, the
// stable LSD radix sort of (key, original index) and the gather of every
// particle array into key order.
//
// Keys: q_a = min(floor((x_a - lo_a) * S), 2^21 - 1), S = 2^21 / L, with L the
// largest extent of the root box (1 if 0); key bit 3b+2/3b+1/3b = bit b of
// q_x/q_y/q_z.  The subtraction and product are done with _rn intrinsics so
// that no multiply-add contraction changes a key.
#include <algorithm>

#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr int kBoxThreads = 256;

// Order-preserving map of a finite double's bits to an unsigned integer
// (negative values: all bits flipped; others: the sign bit set), so that the
// box's min/max are integer comparisons (the FP64 ones run at 1/64 of the
// FP32 rate here).  -0 orders below +0; the value selected is exact either way.
__device__ __forceinline__ unsigned long long ord_of(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double val_of(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

__device__ __forceinline__ void warp_minmax(unsigned long long& mn, unsigned long long& mx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
}

// Per-block min/max of each axis of one patch -> 6 partials per block
// {mn x,y,z, mx x,y,z}.  Without a block map: patch blockIdx.y, its
// gridDim.x blocks, partials at q * gridDim.x + block.  With one (several
// patches of uneven sizes): block b works on patch map[b].x as its map[b].y-th
// of poff[q + 1] - poff[q] blocks (blocks in proportion to the patch sizes),
// partials at b.
__global__ void k_box_partial(const double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ z, const int64_t* __restrict__ off,
                              const uint2* __restrict__ map, const int* __restrict__ poff,
                              unsigned long long* __restrict__ part, int* status) {
    __shared__ unsigned long long s[6][kBoxThreads / 32];
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    int q, j, nbq;
    int64_t slot;
    if (map) {
        const uint2 e = map[blockIdx.x];
        q = (int)e.x;
        j = (int)e.y;
        nbq = poff[q + 1] - poff[q];
        slot = blockIdx.x;
    } else {
        q = blockIdx.y;
        j = blockIdx.x;
        nbq = gridDim.x;
        slot = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    }
    const int64_t e = off[q + 1];
    for (int64_t i = off[q] + (int64_t)j * blockDim.x + threadIdx.x; i < e; i += (int64_t)nbq * blockDim.x) {
        const double v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(v[a]);
            bad |= ((b >> 52) & 0x7ffu) == 0x7ffu;  // infinity or NaN
            const unsigned long long k = ord_of(v[a]);
            mn[a] = min(mn[a], k);
            mx[a] = max(mx[a], k);
        }
    }
    if (bad) atomicOr(status, kStatNonFinite);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        warp_minmax(mn[a], mx[a]);
        if (lane == 0) {
            s[a][w] = mn[a];
            s[3 + a][w] = mx[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        unsigned long long r = s[threadIdx.x][0];
        for (int k = 1; k < kBoxThreads / 32; ++k)
            r = threadIdx.x < 3 ? min(r, s[threadIdx.x][k]) : max(r, s[threadIdx.x][k]);
        part[6 * slot + threadIdx.x] = r;  // (as the ordered integer; a block with no particle keeps the identity)
    }
}

// box of patch q = blockIdx.x from its partials (nb per patch, or those of
// blocks poff[q] .. poff[q + 1] - 1): {lo_x, lo_y, lo_z, L, S} at box + 8 q.
// Cylindrical frame (cyl): every particle must be off the axis (r > 0), else
// kStatAxis.
__global__ void k_box_final(const unsigned long long* __restrict__ part_all, int nb, const int* __restrict__ poff,
                            double* box_all, int cyl, int* status) {
    const unsigned long long* part = part_all + 6 * (poff ? (int64_t)poff[blockIdx.x] : (int64_t)blockIdx.x * nb);
    if (poff) nb = poff[blockIdx.x + 1] - poff[blockIdx.x];
    double* box = box_all + 8 * blockIdx.x;
    __shared__ double r[6];
    if (threadIdx.x < 6) {
        unsigned long long v = part[threadIdx.x];
        for (int b = 1; b < nb; ++b)
            v = threadIdx.x < 3 ? min(v, part[6 * b + threadIdx.x]) : max(v, part[6 * b + threadIdx.x]);
        r[threadIdx.x] = val_of(v);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ext = 0.0;
        for (int a = 0; a < 3; ++a) {
            box[a] = r[a];
            double e = __dsub_rn(r[3 + a], r[a]);
            if (e > ext) ext = e;
        }
        double L = ext > 0.0 ? ext : 1.0;
        box[3] = L;
        box[4] = __ddiv_rn(2097152.0, L);
        if (cyl && !(r[1] > 0.0)) atomicOr(status, kStatAxis);
    }
}

// Sec. 4.3: tree coordinates (phi, r, z) for a ring, phi and r as FP32
// numbers (a tree coordinate only has to place a particle within its key
// cell, 2^-21 of the box; the walk's contact clause has a margin for their
// error).  x, y rounded to FP32; phi from atan of the octant-reduced ratio,
// itself reduced to [0, tan(pi/12)] with
// atan(t) = pi/6 + atan((sqrt(3) t - 1) / (t + sqrt(3))) and summed as the
// Taylor series to u^11 (truncation below 3e-9 rad); r = sqrt(x^2 + y^2).
// Every operation is an IEEE-rounded FP32 +, -, *, / or sqrt in a fixed
// order, so phi is a deterministic function of (x, y), within 1e-6 rad of
// the true angle.
__device__ __forceinline__ float atan01(float t) {
    const float sqrt3 = 1.7320508075688772f, tan15 = 0.2679491924311227f, pi6 = 0.5235987755982988f;
    float base = 0.0f, u = t;
    if (t > tan15) {
        u = __fdiv_rn(__fsub_rn(__fmul_rn(t, sqrt3), 1.0f), __fadd_rn(t, sqrt3));
        base = pi6;
    }
    const float u2 = __fmul_rn(u, u);
    float p = -1.0f / 11.0f;
    p = __fadd_rn(__fmul_rn(p, u2), 1.0f / 9.0f);
    p = __fadd_rn(__fmul_rn(p, u2), -1.0f / 7.0f);
    p = __fadd_rn(__fmul_rn(p, u2), 1.0f / 5.0f);
    p = __fadd_rn(__fmul_rn(p, u2), -1.0f / 3.0f);
    p = __fadd_rn(__fmul_rn(p, u2), 1.0f);
    return __fadd_rn(base, __fmul_rn(u, p));
}

__global__ void k_cyl(const double* __restrict__ x, const double* __restrict__ y, int64_t n,
                      double* __restrict__ phi, double* __restrict__ r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float X = __double2float_rn(x[i]), Y = __double2float_rn(y[i]);
    const float ax = fabsf(X), ay = fabsf(Y);
    const float mx = ax > ay ? ax : ay, mn = ax > ay ? ay : ax;
    float a = 0.0f;
    if (mx != 0.0f) {
        a = atan01(__fdiv_rn(mn, mx));
        if (ay > ax) a = __fsub_rn(1.5707963267948966f, a);
        if (X < 0.0f) a = __fsub_rn(3.141592653589793f, a);
        if (Y < 0.0f) a = __fsub_rn(6.283185307179586f, a);
    }
    phi[i] = (double)a;
    r[i] = (double)__fsqrt_rn(__fadd_rn(__fmul_rn(X, X), __fmul_rn(Y, Y)));
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & kQMax;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// min(max(floor((v - lo) * S), 0), 2^21 - 1) with one FP64 subtraction, one
// product and one truncating conversion (truncation = floor for t >= 0); the
// clamps read the sign and the exponent of t.
__device__ __forceinline__ uint32_t quantise(double v, double lo, double S) {
    const double t = __dmul_rn(__dsub_rn(v, lo), S);
    const unsigned long long b = (unsigned long long)__double_as_longlong(t);
    if (b >> 63) return 0u;                                         // t < 0 (or -0)
    if (((b >> 52) & 0x7ffu) >= 1023u + kLevels) return kQMax;      // t >= 2^21 (infinities and NaN too)
    return min(__double2uint_rz(t), kQMax);
}

// Keys of every particle on its patch's grid (patch by binary search of the
// offsets); idx = the particle's index.
__global__ void k_keys(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, int64_t n, const int64_t* __restrict__ off, int np,
                       const double* __restrict__ boxes, uint64_t* __restrict__ key, uint32_t* __restrict__ idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q = 0;
    for (int lo = 0, hi = np - 1; lo < hi;) {  // last patch starting at or before i
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i)
            lo = q = mid;
        else
            hi = mid - 1;
    }
    const double* box = boxes + 8 * q;
    const double S = box[4];
    uint32_t qx = quantise(x[i], box[0], S), qy = quantise(y[i], box[1], S),
             qz = quantise(z[i], box[2], S);
    key[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    idx[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, passes over bits [8p, 8p+8).  Per pass:
//   upsweep   per-tile digit histogram, stored digit-major hist[d * ntiles + t]
//   scan      exclusive scan of hist -> global start of (digit, tile)
//   downsweep stable in-tile ranking (warp match + per-warp counters), local
//             reorder through shared memory, coalesced scatter.
// Stability: ranks follow (tile, warp, round, lane) = input order.
//
// Several patches (independent particle sets, each sorted on its own): tiles
// never straddle a patch, and the histogram of patch p is stored as its own
// digit-major block after those of patches 0..p-1, so the one scan orders
// the output by (patch, digit, tile).  tmeta holds per tile {first key, key
// count, first tile of its patch, tile count of its patch}; NULL means one
// patch cut into uniform tiles.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                       // per lane
constexpr int kSortTile = kSortThreads * kSortItems; // 4096
constexpr int kRadix = 256;

struct TileInfo {
    int64_t start;  // first key of the tile
    int cnt;        // keys in the tile
    int64_t hbase;  // histogram slot of (digit 0, this tile)
    int nt;         // tile count of the tile's patch (histogram stride)
};

__device__ __forceinline__ TileInfo tile_info(const uint32_t* __restrict__ tmeta, int64_t n, int ntiles) {
    const int t = blockIdx.x;
    TileInfo ti;
    if (tmeta) {
        const uint4 m = reinterpret_cast<const uint4*>(tmeta)[t];
        ti.start = m.x;
        ti.cnt = (int)m.y;
        ti.hbase = (int64_t)kRadix * m.z + (t - (int)m.z);
        ti.nt = (int)m.w;
    } else {
        ti.start = (int64_t)t * kSortTile;
        const int64_t r = n - ti.start;
        ti.cnt = (int)(r < kSortTile ? r : kSortTile);
        ti.hbase = t;
        ti.nt = ntiles;
    }
    return ti;
}

__global__ void k_digit_hist(const uint64_t* __restrict__ key, int64_t n, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[8][kRadix];
    for (int i = threadIdx.x; i < 8 * kRadix; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = key[i];
#pragma unroll
        for (int p = 0; p < 8; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 0xff], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 8 * kRadix; i += blockDim.x)
        if ((&h[0][0])[i]) atomicAdd(&hist[i], (&h[0][0])[i]);
}

__global__ void __launch_bounds__(kSortThreads) k_upsweep(const uint64_t* __restrict__ key, int64_t n,
                                                         int shift, uint32_t* __restrict__ hist,
                                                         int ntiles, const uint32_t* __restrict__ tmeta) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const TileInfo ti = tile_info(tmeta, n, ntiles);
#pragma unroll 4
    for (int k = 0; k < kSortItems; ++k) {
        const int r = k * kSortThreads + threadIdx.x;
        if (r < ti.cnt) atomicAdd(&h[(key[ti.start + r] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[ti.hbase + (int64_t)threadIdx.x * ti.nt] = h[threadIdx.x];
}

struct DownSmem {
    uint32_t whist[kSortWarps][kRadix];
    uint32_t tstart[kRadix];
    uint32_t goff[kRadix];
    uint32_t wtot[kSortWarps];
    uint64_t skey[kSortTile];
    uint32_t sidx[kSortTile];
};

__global__ void __launch_bounds__(kSortThreads) k_downsweep(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ iin, int64_t n, int shift,
    const uint32_t* __restrict__ offs, int ntiles, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ iout, const uint32_t* __restrict__ tmeta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DownSmem& S = *reinterpret_cast<DownSmem*>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&S.whist[0][0])[i] = 0;
    const TileInfo ti = tile_info(tmeta, n, ntiles);
    S.goff[threadIdx.x] = offs[ti.hbase + (int64_t)threadIdx.x * ti.nt];
    __syncthreads();

    const int64_t tbase = ti.start, tend = ti.start + ti.cnt;
    const int64_t wbase = tbase + (int64_t)w * (32 * kSortItems);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t kr[kSortItems];
    uint32_t ir[kSortItems], lr[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t pos = wbase + r * 32 + lane;
        bool valid = pos < tend;
        uint64_t k = valid ? kin[pos] : 0;
        uint32_t d = valid ? (uint32_t)((k >> shift) & 0xff) : 0x100u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && valid) {
            old = S.whist[w][d];
            S.whist[w][d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        kr[r] = k;
        ir[r] = valid ? iin[pos] : 0u;
        lr[r] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive over warps; tile total; exclusive over digits
    {
        const int d = threadIdx.x;  // kSortThreads == kRadix
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ++ww) {
            uint32_t t = S.whist[ww][d];
            S.whist[ww][d] = run;
            run += t;
        }
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) S.wtot[w] = x;
        __syncthreads();
        uint32_t add = 0;
        for (int ww = 0; ww < w; ++ww) add += S.wtot[ww];
        S.tstart[d] = add + x - run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t pos = wbase + r * 32 + lane;
        if (pos < tend) {
            uint32_t d = (uint32_t)((kr[r] >> shift) & 0xff);
            uint32_t p = S.tstart[d] + S.whist[w][d] + lr[r];
            S.skey[p] = kr[r];
            S.sidx[p] = ir[r];
        }
    }
    __syncthreads();
    const int tn = ti.cnt;
    for (int q = threadIdx.x; q < tn; q += kSortThreads) {
        uint64_t k = S.skey[q];
        uint32_t d = (uint32_t)((k >> shift) & 0xff);
        uint64_t g = (uint64_t)S.goff[d] + (uint64_t)(q - S.tstart[d]);
        kout[g] = k;
        iout[g] = S.sidx[q];
    }
}

// All particle arrays (8-byte elements) gathered into key order in one pass:
// the permutation is read once and every array's load is in flight at once;
// dst[a] = scratch + a n (copied back by the caller).
struct Gather8 {
    const unsigned long long* src[8];
    int na;
};

__global__ void k_gather_all(Gather8 G, unsigned long long* __restrict__ scratch, const uint32_t* __restrict__ perm,
                             int64_t n, int* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    if (j >= n) {
        atomicOr(status, kStatBounds);
        return;
    }
    unsigned long long v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
        if (a < G.na) v[a] = G.src[a][j];
#pragma unroll
    for (int a = 0; a < 8; ++a)
        if (a < G.na) scratch[(int64_t)a * n + i] = v[a];
}

}  // namespace

// Root box and keys of each patch (one patch: the whole set).  idx holds
// global particle indices.
int stage_keys(Ctx* c, const bh_particles* p) {
    const int64_t n = c->n;
    const int nbmax = c->num_sms * 4;
    for (int b = 0; b < 2; ++b) {
        BH_TRY(grow(c, c->key[b], (size_t)n, "keys"));
        BH_TRY(grow(c, c->idx[b], (size_t)n, "sort indices"));
    }
    // tree coordinates: (x, y, z), or (phi, r, z) in the cylindrical frame
    const double *cx = p->x, *cy = p->y;
    if (c->prm.key_frame == 1) {
        BH_TRY(grow(c, c->cyl, 2 * (size_t)n, "cylindrical coordinates"));
        k_cyl<<<blocks_for(n, 256), 256, 0, c->stream>>>(p->x, p->y, n, c->cyl.p, c->cyl.p + n);
        BH_LAUNCH(c);
        cx = c->cyl.p;
        cy = c->cyl.p + n;
    }
    // all patches at once: blocks for the boxes (in proportion to the patch
    // sizes when there are several), then one pass for the keys
    const int np = c->n_patches;
    if (np > 1) {
        const int nbt = c->n_box_blocks;
        BH_TRY(grow(c, c->box_part, 6 * (size_t)nbt, "box partials"));
        k_box_partial<<<nbt, kBoxThreads, 0, c->stream>>>(cx, cy, p->z, c->d_off.p, c->box_map.p, c->box_poff.p,
                                                          c->box_part.p, c->d_status);
        BH_LAUNCH(c);
        k_box_final<<<np, 32, 0, c->stream>>>(c->box_part.p, 0, c->box_poff.p, c->d_box, c->prm.key_frame == 1,
                                              c->d_status);
        BH_LAUNCH(c);
    } else {
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(nbmax, blocks_for(n, 4 * kBoxThreads)));
        BH_TRY(grow(c, c->box_part, 6 * (size_t)nb, "box partials"));
        k_box_partial<<<nb, kBoxThreads, 0, c->stream>>>(cx, cy, p->z, c->d_off.p, nullptr, nullptr,
                                                         c->box_part.p, c->d_status);
        BH_LAUNCH(c);
        k_box_final<<<1, 32, 0, c->stream>>>(c->box_part.p, nb, nullptr, c->d_box, c->prm.key_frame == 1,
                                             c->d_status);
        BH_LAUNCH(c);
    }
    k_keys<<<blocks_for(n, 256), 256, 0, c->stream>>>(cx, cy, p->z, n, c->d_off.p, np, c->d_box, c->key[0].p,
                                                      c->idx[0].p);
    BH_LAUNCH(c);
    c->key_cur = 0;
    return BH_OK;
}

int stage_sort(Ctx* c) {
    const int64_t n = c->n;
    const uint32_t* tmeta = c->n_patches > 1 ? c->tile_meta.p : nullptr;
    const int ntiles = c->n_patches > 1 ? (int)c->n_tiles : (int)((n + kSortTile - 1) / kSortTile);
    BH_TRY(grow(c, c->digit_hist, 8 * kRadix, "digit histogram"));
    BH_TRY(grow(c, c->sort_hist, (size_t)kRadix * ntiles, "sort histogram"));
    BH_CUDA(c, cudaMemsetAsync(c->digit_hist.p, 0, 8 * kRadix * sizeof(uint32_t), c->stream));
    // passes whose digit is the same for every key leave the order as it is
    // and are skipped (a device-sized build runs all eight: nothing is read
    // back; the sort is stable, so the result is the same)
    uint32_t h[8 * kRadix] = {};
    if (!c->dev_build) {
        k_digit_hist<<<c->num_sms * 2, 256, 0, c->stream>>>(c->key[c->key_cur].p, n, c->digit_hist.p);
        BH_LAUNCH(c);
        BH_CUDA(c, cudaMemcpyAsync(h, c->digit_hist.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    const int smem = (int)sizeof(DownSmem);
    if (c->sort_attr_device != c->device) {  // once per device
        BH_CUDA(c, cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        c->sort_attr_device = c->device;
    }
    for (int pass = 0; pass < 8; ++pass) {
        bool trivial = false;
        for (int d = 0; d < kRadix; ++d)
            if ((int64_t)h[pass * kRadix + d] == n) trivial = true;
        if (trivial) continue;  // every key has the same digit: order unchanged
        const int shift = 8 * pass, a = c->key_cur, b = 1 - a;
        k_upsweep<<<ntiles, kSortThreads, 0, c->stream>>>(c->key[a].p, n, shift, c->sort_hist.p, ntiles, tmeta);
        BH_LAUNCH(c);
        BH_TRY(scan_u32(c, c->sort_hist.p, c->sort_hist.p, (int64_t)kRadix * ntiles, nullptr));
        k_downsweep<<<ntiles, kSortThreads, smem, c->stream>>>(c->key[a].p, c->idx[a].p, n, shift,
                                                               c->sort_hist.p, ntiles, c->key[b].p,
                                                               c->idx[b].p, tmeta);
        BH_LAUNCH(c);
        c->key_cur = b;
    }
    return BH_OK;
}

int stage_permute(Ctx* c, bh_particles* p) {
    const int64_t n = c->n;
    BH_TRY(grow(c, c->pscratch, 8 * (size_t)n, "particle scratch"));
    unsigned long long* arrs[8] = {(unsigned long long*)p->x,  (unsigned long long*)p->y,
                                   (unsigned long long*)p->z,  (unsigned long long*)p->vx,
                                   (unsigned long long*)p->vy, (unsigned long long*)p->vz,
                                   (unsigned long long*)p->m,  (unsigned long long*)p->id};
    const uint32_t* perm = c->idx[c->key_cur].p;
    Gather8 G;
    unsigned long long* dst[8];
    G.na = 0;
    for (int a = 0; a < 8; ++a)
        if (arrs[a]) {
            dst[G.na] = arrs[a];
            G.src[G.na++] = arrs[a];
        }
    unsigned long long* scratch = (unsigned long long*)c->pscratch.p;
    k_gather_all<<<blocks_for(n, 256), 256, 0, c->stream>>>(G, scratch, perm, n, c->d_status);
    BH_LAUNCH(c);
    for (int a = 0; a < G.na; ++a)
        BH_CUDA(c, cudaMemcpyAsync(dst[a], scratch + (int64_t)a * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                   c->stream));
    return BH_OK;
}

// Sort tiles of the patches: 4 words per tile (see TileInfo).
int64_t sort_tiles_for(const std::vector<int64_t>& off, std::vector<uint32_t>* meta) {
    int64_t t = 0;
    for (size_t q = 0; q + 1 < off.size(); ++q) {
        const int64_t np = off[q + 1] - off[q], nt = (np + kSortTile - 1) / kSortTile, t0 = t;
        for (int64_t u = 0; u < nt; ++u, ++t) {
            if (meta) {
                const int64_t st = off[q] + u * kSortTile, r = off[q + 1] - st;
                meta->push_back((uint32_t)st);
                meta->push_back((uint32_t)(r < kSortTile ? r : kSortTile));
                meta->push_back((uint32_t)t0);
                meta->push_back((uint32_t)nt);
            }
        }
    }
    return t;
}

// Context-free form of stage_sort for callers that supply every buffer: all
// eight passes run (no host read-back of the digit histogram, so nothing here
// synchronises), ending in (keys, idx) again.  idx is set to 0..n-1 first.
int64_t sort_scratch_words(int64_t n) {
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    return kRadix * ntiles + scan_sums_count(kRadix * ntiles);
}

cudaError_t sort_setup_device() {
    return cudaFuncSetAttribute(k_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DownSmem));
}

namespace {
__global__ void k_iota(uint32_t* __restrict__ idx, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) idx[i] = (uint32_t)i;
}
}  // namespace

cudaError_t sort_pairs_with(cudaStream_t s, uint64_t* keys, uint32_t* idx, uint64_t* ktmp, uint32_t* itmp,
                            int64_t n, uint32_t* scratch) {
    if (n <= 0) return cudaSuccess;
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    uint32_t* hist = scratch;
    uint32_t* sums = scratch + (int64_t)kRadix * ntiles;
    k_iota<<<blocks_for(n, 256), 256, 0, s>>>(idx, n);
    uint64_t* kb[2] = {keys, ktmp};
    uint32_t* ib[2] = {idx, itmp};
    for (int pass = 0; pass < 8; ++pass) {
        const int a = pass & 1, b = 1 - a;
        k_upsweep<<<ntiles, kSortThreads, 0, s>>>(kb[a], n, 8 * pass, hist, ntiles, nullptr);
        cudaError_t e = scan_u32_with(s, hist, hist, (int64_t)kRadix * ntiles, sums);
        if (e != cudaSuccess) return e;
        k_downsweep<<<ntiles, kSortThreads, sizeof(DownSmem), s>>>(kb[a], ib[a], n, 8 * pass, hist, ntiles,
                                                                   kb[b], ib[b], nullptr);
    }
    return cudaGetLastError();
}

}  // namespace bh
