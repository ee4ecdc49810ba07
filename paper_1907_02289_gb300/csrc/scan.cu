// scan.cu -- device-wide exclusive prefix sums (reduce, scan block sums,
// scan tiles with offsets).  Used for radix-sort digit offsets, octree child
// offsets, group compaction and list offsets.
#include <algorithm>

#include "bh_internal.cuh"

namespace bh {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <typename T>
__device__ T block_exclusive(T v, T* warp_tot, T* block_total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = (lane < kThreads / 32) ? warp_tot[lane] : T(0);
        T s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_tot[lane] = s - t;
        if (lane == kThreads / 32 - 1) *block_total = s;
    }
    __syncthreads();
    T r = warp_tot[w] + x - v;
    __syncthreads();
    return r;
}

// Element count: n, or the device count *dn capped at n (device-sized scans,
// whose grid is fixed when they are issued; blocks then stride over tiles).
__device__ __forceinline__ int64_t count_of(int64_t n, const unsigned long long* dn) {
    if (!dn) return n;
    const unsigned long long v = *dn;
    return v < (unsigned long long)n ? (int64_t)v : n;
}

template <typename T>
__global__ void k_reduce(const T* __restrict__ in, int64_t n, const unsigned long long* dn, T* __restrict__ sums) {
    __shared__ T wt[kThreads / 32];
    __shared__ T tot;
    n = count_of(n, dn);
    const int64_t nt = (n + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t base = tile * kTile;
        T s = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
            if (i < n) s += in[i];
        }
        block_exclusive<T>(s, wt, &tot);
        if (threadIdx.x == 0) sums[tile] = tot;
    }
}

// One block: exclusive scan of the block sums in place; total to *d_total.
template <typename T>
__global__ void k_scan_sums(T* sums, int64_t n, const unsigned long long* dn, unsigned long long* d_total) {
    __shared__ T wt[kThreads / 32];
    __shared__ T tot;
    n = count_of(n, dn);
    const int64_t nb = (n + kTile - 1) / kTile;
    T carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kThreads) {
        int64_t i = b0 + threadIdx.x;
        T v = (i < nb) ? sums[i] : T(0);
        T e = block_exclusive<T>(v, wt, &tot);
        if (i < nb) sums[i] = carry + e;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && d_total) *d_total = (unsigned long long)carry;
}

// Blocked arrangement: thread t owns items [t*kItems, (t+1)*kItems) of the tile.
template <typename T>
__global__ void k_scan_apply(const T* __restrict__ in, T* __restrict__ out, int64_t n, const unsigned long long* dn,
                             const T* __restrict__ sums) {
    __shared__ T wt[kThreads / 32];
    __shared__ T tot;
    __shared__ T stage[kTile];
    n = count_of(n, dn);
    const int64_t nt = (n + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t base = tile * kTile;
        for (int k = 0; k < kItems; ++k) {
            int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
            stage[k * kThreads + threadIdx.x] = (i < n) ? in[i] : T(0);
        }
        __syncthreads();
        T v[kItems], s = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            v[k] = stage[threadIdx.x * kItems + k];
            s += v[k];
        }
        T e = block_exclusive<T>(s, wt, &tot) + sums[tile];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            stage[threadIdx.x * kItems + k] = e;
            e += v[k];
        }
        __syncthreads();
        for (int k = 0; k < kItems; ++k) {
            int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
            if (i < n) out[i] = stage[k * kThreads + threadIdx.x];
        }
        __syncthreads();
    }
}

// dn == nullptr: n elements, one tile per block.  Otherwise *dn elements
// (read on the device, at most n) over a grid fixed here.
template <typename T>
int scan_impl(Ctx* c, const T* in, T* out, int64_t n, unsigned long long* d_total, const unsigned long long* dn) {
    if (n <= 0) {
        if (d_total) BH_CUDA(c, cudaMemsetAsync(d_total, 0, sizeof(unsigned long long), c->stream));
        return BH_OK;
    }
    const int64_t nb = (n + kTile - 1) / kTile;
    BH_TRY(grow(c, c->scan_tmp, (size_t)nb * sizeof(T), "scan block sums"));
    T* sums = (T*)c->scan_tmp.p;
    const unsigned grid = dn ? (unsigned)std::min<int64_t>(nb, 4 * (int64_t)c->num_sms) : (unsigned)nb;
    k_reduce<T><<<grid, kThreads, 0, c->stream>>>(in, n, dn, sums);
    BH_LAUNCH(c);
    k_scan_sums<T><<<1, kThreads, 0, c->stream>>>(sums, n, dn, d_total);
    BH_LAUNCH(c);
    k_scan_apply<T><<<grid, kThreads, 0, c->stream>>>(in, out, n, dn, sums);
    BH_LAUNCH(c);
    return BH_OK;
}

}  // namespace

int scan_u32(Ctx* c, const uint32_t* in, uint32_t* out, int64_t n, unsigned long long* d_total,
             const unsigned long long* dn) {
    return scan_impl<uint32_t>(c, in, out, n, d_total, dn);
}
int scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, unsigned long long* d_total,
             const unsigned long long* dn) {
    return scan_impl<int64_t>(c, in, out, n, d_total, dn);
}

// Context-free form of scan_u32 over caller-provided block sums (at least
// scan_sums_count(n) words); launches only, errors from cudaGetLastError.
int64_t scan_sums_count(int64_t n) { return n <= 0 ? 0 : (n + kTile - 1) / kTile; }

cudaError_t scan_u32_with(cudaStream_t s, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* sums) {
    if (n <= 0) return cudaSuccess;
    const int64_t nb = scan_sums_count(n);
    k_reduce<uint32_t><<<(unsigned)nb, kThreads, 0, s>>>(in, n, nullptr, sums);
    k_scan_sums<uint32_t><<<1, kThreads, 0, s>>>(sums, n, nullptr, nullptr);
    k_scan_apply<uint32_t><<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, nullptr, sums);
    return cudaGetLastError();
}

}  // namespace bh
