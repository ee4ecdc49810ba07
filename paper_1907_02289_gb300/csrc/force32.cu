// force32.cu -- the FP32 group-relative force kernel (Sec. 4.7: positions
// shifted to an origin inside the group, then single precision).  Origin:
// the centre of mass of the group node, taken from the node's FP32 hi/lo
// record.
//
// Shift: every FP64 coordinate is split once per evaluation into FP32 hi/lo
// parts, so no FP64 arithmetic (1/64 of the FP32 rate on this GPU) runs per
// list entry.  List particles and the group's particles are held relative to
// the origin as FP32 hi/lo pairs, and the separation of a pair is formed as
// (x_hi,j - x_hi,i) + (x_lo,j - x_lo,i): exact to an FP32 rounding of the
// separation itself, however wide the group is.  List cells, which the
// opening test keeps at least a cell size away, use the hi part alone, and
// so do "far" list particles (beyond contact reach and at least an eighth of
// the group's largest side away; the list expansion puts them after the
// near ones): their separation is the difference of the two rounded FP32
// coordinates, as in Sec. 4.7, correct to about 30 FP32 unit roundings of
// itself at most at that distance, and they need no contact test.
//
// Gravity inside r_coll (Eq. 1) is G m_j r / (r_coll^2 + eps^2)^(3/2), so
// max(r^2, r_coll^2) + eps^2 in the fast loop gives it for every pair (and
// 0 for i = j).  Pairs that may be in contact are queued per warp and
// appended to a global list; a separate FP64 pass adds their contact term
// of Eq. (1) in the oracle's operation order (the r <= r_coll decision
// included), with every lane busy -- FP64 inside the warp loop would leave
// 31 lanes idle at 1/64 of the FP32 rate -- summing each particle's terms
// in fixed point so that the result does not depend on the list's order.
//
// Summation: FP32 partial sums per tile (even and odd list entries apart),
// folded after every tile into a compensated (TwoSum) hi/lo accumulator in
// shared memory.
//
// Conditioning and refinement: the fold also sums the squares of the tile
// partial sums.  The FP32 error of a_i (rounding of each term and of the
// partial sums, both random in sign) grows with the root of that sum, not
// with |a_i|, so where the pulls on a particle nearly cancel its relative
// error grows without bound.  A particle with |a_i| below 0.12 G times that
// root (about 0.3% of a ring's particles, measured) is queued, and a second
// kernel evaluates it again over the same lists in df arithmetic (pairs of
// FP32 numbers, dfloat.cuh), from the hi/lo coordinates and masses, and
// replaces a_i.
//
// Mapping: one warp per group.  A group of n_i = 32 R + t particles gives
// every lane R i-slots; the t remaining particles go to a "tail" slot shared
// by J = 32 / T lanes (T = t rounded up to a power of two) that split the
// list between them, so a 65-particle group costs 2 + 1/32 slots rather
// than 3.  List entries are staged in pairs in shared memory and broadcast,
// and the pair (j, j+1) is evaluated with packed f32x2 instructions (FADD2,
// FFMA2, FMUL2) against the i-particle held as (x_i, x_i), which halves the
// issue slots per interaction.  The next tile is gathered with cp.async
// while the current one is evaluated.  Groups larger than the i-chunk (at
// most 96) are evaluated chunk by chunk.  The group's own particles are
// evaluated first in a phase that excludes i = j; the expanded list holds
// only the other particles.
//
// Scheduling: groups are taken in order of size class (warps running side
// by side execute the same code), by decreasing estimated cost within a
// class, optionally within windows of consecutive groups; the grid is one
// warp per group, or persistent (resident blocks only) with warps taking
// groups round robin or from an atomic ticket counter.  Warps per block and
// the i-chunk are runtime settings; the compile-time options below exist for
// experiments.
#include <algorithm>
#include <cmath>

#include "dfloat.cuh"
#include "force_common.cuh"

namespace bh {
namespace {

#ifndef BH_F32_MAXW
#define BH_F32_MAXW 8  // most warps per block (the register budget is sized for 2 such blocks per SM)
#endif
#ifndef BH_F32_UNROLL
#define BH_F32_UNROLL 1  // list pairs per iteration of the particle loop
#endif
#ifndef BH_F32_PCUNROLL
#define BH_F32_PCUNROLL 1  // list pairs per iteration of the cell loop
#endif
#ifndef BH_F32_MAXR
#define BH_F32_MAXR 3  // most full i-slots per lane (chunks of up to 32 x this particles)
#endif
#ifndef BH_F32_TILE
#define BH_F32_TILE 1  // list particles per tile = 64 x this, list cells = 32 x this
#endif
#ifndef BH_REFINE_K
// refinement threshold: |a_i| < K G sqrt(sum of squared tile partial sums);
// measured on the 2^24 and 2^26 rings and the 64 patches, it sends about 0.3%
// of the particles to the refinement and leaves the others below 6e-6
#define BH_REFINE_K 0.12
#endif
constexpr int kTileJ = 64 * BH_F32_TILE;  // list particles per tile (2 per lane per 64)
constexpr int kTileC = 32 * BH_F32_TILE;  // list cells per tile (1 per lane per 32)
constexpr int kSlots = 3;                 // i-slots per lane (full slots + tail)
constexpr int kUnrollPP = BH_F32_UNROLL, kUnrollPC = BH_F32_PCUNROLL;
constexpr int kQueueCap = 32 + 2 * kSlots * 32;
constexpr uint32_t kNone = 0xffffffffu;

// Pair-term modes: contact candidates detected (r_coll > 0); plain (no
// contact, r_coll^2 + eps^2 > 0); mask (r_coll = eps = 0: coincident pairs
// masked out explicitly); contact without softening (r_coll > 0, eps = 0,
// which saves the + eps^2 of every pair).
constexpr int kContact = 0, kPlain = 1, kMask = 2, kContact0 = 3;
__host__ __device__ constexpr bool has_contact(int mode) { return mode == kContact || mode == kContact0; }

struct __align__(16) JPair {  // two list particles relative to the origin (hi/lo)
    float2 x, y, z, m, xl, yl, zl, pad;
};
struct CPair {  // two cells: centre relative to the origin, mass, negated quadrupole
    float2 x, y, z, m, qxx, qxy, qxz, qyy, qyz, qzz;
};

struct Smem32 {
    union {
        struct {
            JPair jp[kTileJ / 2];
            uint32_t jid[kTileJ];
        } p;
        CPair cp[kTileC / 2];
    } t;
    union {  // raw gathered data of the next tile (filled by cp.async)
        struct {
            float4 h[kTileJ], l[kTileJ];
        } p;
        float4 c[kTileC][3];
    } raw;
    uint32_t raw_id[kTileJ];
    uint32_t q_i[kQueueCap];   // contact candidates (i, j) waiting for the global list
    uint32_t q_j[kQueueCap];
    float2 acc[32 * kSlots][3];  // compensated sums (G-free): (hi, lo), one 8-byte access each
    float abnd[32 * kSlots];    // sum over folds of squared tile partial sums (conditioning of the sum)
    uint8_t hasc[32 * kSlots];  // the slot's particle has a contact candidate
};

struct Args {
    int64_t ng;
    const unsigned long long* dng;  // device group count (device-sized list builds; NULL: ng)
    const unsigned long long* abort;  // device-sized build: nonzero overflow bits skip the launch
    const int32_t* order;  // processing order of the groups (NULL: list order)
    const int32_t* groups;
    const uint32_t* begin;
    const uint32_t* end;
    const int64_t* jj_off;
    const int64_t* jj_mid;  // per group index of the first far list particle (NULL: none)
    const uint32_t* JJ;
    const int64_t* pc_off;
    const int32_t* C;
    const float4* phi;
    const float4* plo;
    const float4* cell32;
    const double *x, *y, *z;
    double *ax, *ay, *az;
    uint2* contacts;               // (i, j) pairs for the FP64 contact pass
    unsigned long long* ncontact;  // its counter
    int64_t contact_cap;
    uint32_t n;
    int64_t nn;
    int* status;
    ForceParams fp;
    float floor2;   // r_coll^2 + eps^2 (or eps^2)
    float rc2chk;   // r^2 below this (FP32) may be a contact: r_coll^2 (1 + 1e-5)
    bool add_central;
    // schedule: warps take list slots slot0, slot0 + stride, ... (grid or
    // persistent static), or draw them from *ticket (persistent dynamic)
    int chunk;                     // largest i-chunk (32, 64 or 96 particles)
    unsigned long long* ticket;    // NULL: static
    unsigned long long* warp_time; // optional: per warp (start, end) %globaltimer
    // refinement: particle i of list slot k is queued as (i, k) when
    // |a_i| < kref * G * sqrt(sum over tiles of the squared tile partial sums)
    uint2* refine;
    unsigned long long* nrefine;
    double kref;
    // particles with a contact candidate are judged after the contact pass
    // (the spring can cancel the gravity): their bound and list slot wait here
    float* cbnd;
    uint32_t* cslot;
    unsigned* cflag;
    const double *vx, *vy, *vz, *m;  // FP64 arrays for the refinement's contact terms
};

__device__ __forceinline__ float rel(float hi, float lo, float ohi, float olo) {
    return __fadd_rn(__fsub_rn(hi, ohi), __fsub_rn(lo, olo));
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// (x_hi + x_lo) - (o_hi + o_lo) as an FP32 hi/lo pair.
__device__ __forceinline__ void rel2(float xh, float xl, float oh, float ol, float& rh, float& rl) {
    const float s = __fsub_rn(xh, oh);
    const float v = __fsub_rn(s, xh);
    const float e = __fsub_rn(__fsub_rn(xh, __fsub_rn(s, v)), __fadd_rn(oh, v));  // s + e == xh - oh exactly
    const float t = __fadd_rn(e, __fsub_rn(xl, ol));
    rh = __fadd_rn(s, t);
    rl = __fsub_rn(t, __fsub_rn(rh, s));
}

// Central mass, FP64: r^-1 from the FP32 estimate refined by two Newton
// steps y <- y (3 - r2 y^2) / 2 (each roughly doubles the correct bits).
__device__ __forceinline__ void central_newton(double G_Mc, double x, double y, double z, double* a) {
    const double r2 = fma(x, x, fma(y, y, z * z));
    double yv = (double)rsqrtf((float)r2);
    yv = yv * fma(-0.5 * r2, yv * yv, 1.5);
    yv = yv * fma(-0.5 * r2, yv * yv, 1.5);
    const double f = -G_Mc * (yv * yv * yv);
    a[0] = fma(f, x, a[0]);
    a[1] = fma(f, y, a[1]);
    a[2] = fma(f, z, a[2]);
}

// ---- per-chunk state ------------------------------------------------------
// Slot r (r < R): lane holds particle i0 + 32 r + lane.  Tail slot (r == R):
// lane holds i0 + 32 R + (lane % T) and sees only the list pairs q with
// q % J == lane / T.  Coordinates are stored negated, (-x, -x).
template <int R, bool TAIL>
struct Chunk {
    static constexpr int NS = R + (TAIL ? 1 : 0);
    float2 nh[NS][3], nl[NS][3], g[NS][3];
    uint32_t iv[NS];
    bool vl[NS];
};

// ---- contact candidates ---------------------------------------------------
// Queued pairs go to the global list for the FP64 contact pass.
__device__ __noinline__ void flush_queue(const Args& A, Smem32& S, int& qn, int lane) {
    for (int base = 0; base < qn; base += 32) {
        const int u = base + lane;
        const bool has = u < qn;
        const unsigned msk = __ballot_sync(0xffffffffu, has);
        unsigned long long pos0 = 0;
        if (lane == 0) pos0 = atomicAdd(A.ncontact, (unsigned long long)__popc(msk));
        pos0 = __shfl_sync(0xffffffffu, pos0, 0);
        if (has) {
            const unsigned long long pos = pos0 + lane;
            if ((int64_t)pos < A.contact_cap) A.contacts[pos] = make_uint2(S.q_i[u], S.q_j[u]);
        }
    }
    __syncwarp();
    qn = 0;
}

// Queue the contact candidates of list pair P for slots [r0, r1) (flags
// recomputed here; rare path).  Warp-uniform call.
template <bool SELF, int R, bool TAIL>
__device__ __forceinline__ void queue_pair(const Args& A, Smem32& S, int& qn, const JPair& P, const uint32_t* jid,
                                           const Chunk<R, TAIL>& K, int r0, int r1, bool tail_ok, int lane) {
    constexpr int NS = Chunk<R, TAIL>::NS;
    unsigned bits = 0;
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        if (r < r0 || r >= r1) continue;
        const bool ok = K.vl[r] && ((r < R) || tail_ok);
        float2 d[3];
        d[0] = __fadd2_rn(__fadd2_rn(P.x, K.nh[r][0]), __fadd2_rn(P.xl, K.nl[r][0]));
        d[1] = __fadd2_rn(__fadd2_rn(P.y, K.nh[r][1]), __fadd2_rn(P.yl, K.nl[r][1]));
        d[2] = __fadd2_rn(__fadd2_rn(P.z, K.nh[r][2]), __fadd2_rn(P.zl, K.nl[r][2]));
        const float2 r2 = __ffma2_rn(d[0], d[0], __ffma2_rn(d[1], d[1], __fmul2_rn(d[2], d[2])));
        if (ok && r2.x < A.rc2chk && jid[0] != K.iv[r] && jid[0] != kNone) bits |= 1u << (2 * r);
        if (ok && r2.y < A.rc2chk && jid[1] != K.iv[r] && jid[1] != kNone) bits |= 2u << (2 * r);
    }
    const int c = __popc(bits);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const int total = __shfl_sync(0xffffffffu, x, 31);
    int pos = qn + x - c;
#pragma unroll
    for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (bits & (1u << (2 * r + h))) {
                S.q_i[pos] = K.iv[r];
                S.q_j[pos] = jid[h];
                S.hasc[32 * r + lane] = 1;
                ++pos;
            }
    qn += total;
    __syncwarp();
}

// ---- interaction bodies ------------------------------------------------------
// Particle-particle term of one list pair for one slot (G-free).  Returns
// whether a contact candidate was seen (self excluded when SELF).
template <int MODE, bool SELF>
__device__ __forceinline__ bool pp_body(const Args& A, const JPair& P, const uint32_t* jid, uint32_t i,
                                        const float2 (&nh)[3], const float2 (&nl)[3], float2 (&g)[3]) {
    const float2 dx = __fadd2_rn(__fadd2_rn(P.x, nh[0]), __fadd2_rn(P.xl, nl[0]));
    const float2 dy = __fadd2_rn(__fadd2_rn(P.y, nh[1]), __fadd2_rn(P.yl, nl[1]));
    const float2 dz = __fadd2_rn(__fadd2_rn(P.z, nh[2]), __fadd2_rn(P.zl, nl[2]));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    float2 s2;
    if (MODE == kMask) {
        s2 = r2;
    } else if (MODE == kContact0) {
        s2.x = fmaxf(r2.x, A.floor2);
        s2.y = fmaxf(r2.y, A.floor2);
    } else {
        s2.x = fmaxf(r2.x + A.fp.eps2f, A.floor2);
        s2.y = fmaxf(r2.y + A.fp.eps2f, A.floor2);
    }
    const float2 ri = make_float2(rsqrt_approx(s2.x), rsqrt_approx(s2.y));
    float2 f = __fmul2_rn(__fmul2_rn(P.m, ri), __fmul2_rn(ri, ri));
    if (MODE == kMask) {
        f.x = r2.x > 0.f ? f.x : 0.f;
        f.y = r2.y > 0.f ? f.y : 0.f;
    }
    g[0] = __ffma2_rn(f, dx, g[0]);
    g[1] = __ffma2_rn(f, dy, g[1]);
    g[2] = __ffma2_rn(f, dz, g[2]);
    if (!has_contact(MODE)) return false;
    if (SELF) return (r2.x < A.rc2chk && jid[0] != i) || (r2.y < A.rc2chk && jid[1] != i);
    return r2.x < A.rc2chk || r2.y < A.rc2chk;
}

// Far particle-particle term (G-free): single-float separation, no contact
// test; r > r_coll is certain, so neither the floor nor a mask applies.
__device__ __forceinline__ void pp_far_body(const JPair& P, const float2 (&nh)[3], float2 (&g)[3], float2 eps2) {
    const float2 dx = __fadd2_rn(P.x, nh[0]);
    const float2 dy = __fadd2_rn(P.y, nh[1]);
    const float2 dz = __fadd2_rn(P.z, nh[2]);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
    const float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
    const float2 f = __fmul2_rn(__fmul2_rn(P.m, ri), __fmul2_rn(ri, ri));
    g[0] = __ffma2_rn(f, dx, g[0]);
    g[1] = __ffma2_rn(f, dy, g[1]);
    g[2] = __ffma2_rn(f, dz, g[2]);
}

template <int ORDER>
__device__ __forceinline__ void pc_body(const CPair& Cp, const float2 (&nh)[3], float2 (&g)[3], float2 eps2) {
    const float2 dx = __fadd2_rn(Cp.x, nh[0]);
    const float2 dy = __fadd2_rn(Cp.y, nh[1]);
    const float2 dz = __fadd2_rn(Cp.z, nh[2]);
    const float2 R2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
    const float2 ri = make_float2(rsqrt_approx(R2.x), rsqrt_approx(R2.y));
    const float2 ri2 = __fmul2_rn(ri, ri);
    const float2 ri3 = __fmul2_rn(ri, ri2);
    if (ORDER >= 2) {
        // q = -Q d, dqd = d.(-Q d); a += (M R^2 - 5/2 dqd / R^2) d / R^5 + q / R^5
        const float2 qx = __ffma2_rn(Cp.qxx, dx, __ffma2_rn(Cp.qxy, dy, __fmul2_rn(Cp.qxz, dz)));
        const float2 qy = __ffma2_rn(Cp.qxy, dx, __ffma2_rn(Cp.qyy, dy, __fmul2_rn(Cp.qyz, dz)));
        const float2 qz = __ffma2_rn(Cp.qxz, dx, __ffma2_rn(Cp.qyz, dy, __fmul2_rn(Cp.qzz, dz)));
        const float2 dqd = __ffma2_rn(dx, qx, __ffma2_rn(dy, qy, __fmul2_rn(dz, qz)));
        const float2 ri4 = __fmul2_rn(ri2, ri2);
        const float2 ri5 = __fmul2_rn(ri4, ri);
        const float2 s = __ffma2_rn(__fmul2_rn(dqd, ri2), f2(-2.5f), __fmul2_rn(Cp.m, R2));
        g[0] = __ffma2_rn(ri5, __ffma2_rn(s, dx, qx), g[0]);
        g[1] = __ffma2_rn(ri5, __ffma2_rn(s, dy, qy), g[1]);
        g[2] = __ffma2_rn(ri5, __ffma2_rn(s, dz, qz), g[2]);
    } else {
        const float2 s = __fmul2_rn(Cp.m, ri3);
        g[0] = __ffma2_rn(s, dx, g[0]);
        g[1] = __ffma2_rn(s, dy, g[1]);
        g[2] = __ffma2_rn(s, dz, g[2]);
    }
}

__device__ __forceinline__ void fold(Smem32& S, int s, float2 (&g)[3]) {
    float bnd = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float t = __fadd_rn(g[c].x, g[c].y);
        bnd = __fmaf_rn(t, t, bnd);
        const float2 cur = S.acc[s][c];
        const float hi = cur.x;
        const float s1 = __fadd_rn(hi, t);
        const float bp = __fsub_rn(s1, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s1, bp)), __fsub_rn(t, bp));
        S.acc[s][c] = make_float2(s1, __fadd_rn(cur.y, err));
        g[c] = make_float2(0.f, 0.f);
    }
    S.abnd[s] += bnd;
}

template <int R, bool TAIL>
__device__ __forceinline__ void fold_all(Smem32& S, Chunk<R, TAIL>& K, int lane) {
#pragma unroll
    for (int r = 0; r < Chunk<R, TAIL>::NS; ++r) fold(S, 32 * r + lane, K.g[r]);
}

// ---- staging -------------------------------------------------------------------
// Asynchronous 16-byte global -> shared copies (no registers held while the
// gather is in flight); one commit group per tile, waited for at the top of
// the next tile.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Start the gather of list particle j into raw slot u (kNone: nothing).
__device__ __forceinline__ void gather_particle(const Args& A, Smem32& S, int u, uint32_t j) {
    S.raw_id[u] = j;
    if (j != kNone) {
        cp_async16(&S.raw.p.h[u], &A.phi[j]);
        cp_async16(&S.raw.p.l[u], &A.plo[j]);
    }
}

// Raw slot u -> entry u of the particle tile, relative to the origin as
// hi/lo pairs (padding when !real); FAR: the hi parts (the rounded relative
// coordinates) and the mass only.
template <bool FAR>
__device__ __forceinline__ void put_particle(Smem32& S, int u, bool real, const float (&oh)[3],
                                             const float (&ol)[3]) {
    float ph[3], pl[3], pm;
    if (real && FAR) {  // the rounded relative coordinates only: 3 additions each
        const float4 h = S.raw.p.h[u], l = S.raw.p.l[u];
        ph[0] = rel(h.x, l.x, oh[0], ol[0]);
        ph[1] = rel(h.y, l.y, oh[1], ol[1]);
        ph[2] = rel(h.z, l.z, oh[2], ol[2]);
        pl[0] = pl[1] = pl[2] = 0.f;
        pm = h.w;
    } else if (real) {
        const float4 h = S.raw.p.h[u], l = S.raw.p.l[u];
        rel2(h.x, l.x, oh[0], ol[0], ph[0], pl[0]);
        rel2(h.y, l.y, oh[1], ol[1], ph[1], pl[1]);
        rel2(h.z, l.z, oh[2], ol[2], ph[2], pl[2]);
        pm = h.w;
    } else {  // padding entry: far away, massless
        ph[0] = ph[1] = ph[2] = 1e15f;
        pl[0] = pl[1] = pl[2] = 0.f;
        pm = 0.f;
    }
    float* base = reinterpret_cast<float*>(&S.t.p.jp[u >> 1]);
    const int hh = u & 1;
    base[0 + hh] = ph[0];
    base[2 + hh] = ph[1];
    base[4 + hh] = ph[2];
    base[6 + hh] = pm;
    if (FAR) return;
    base[8 + hh] = pl[0];
    base[10 + hh] = pl[1];
    base[12 + hh] = pl[2];
    S.t.p.jid[u] = real ? S.raw_id[u] : kNone;
}

__device__ __forceinline__ void gather_cell(const Args& A, Smem32& S, int u, int32_t cc, int nrec) {
    if (cc >= 0)
        for (int a = 0; a < nrec; ++a) cp_async16(&S.raw.c[u][a], &A.cell32[3 * (int64_t)cc + a]);
}

__device__ __forceinline__ uint32_t list_index(const Args& A, int64_t p, int64_t j1, uint32_t fallback) {
    if (p >= j1) return kNone;
    uint32_t j = A.JJ[p];
    if (j >= A.n) {
        atomicOr(A.status, kStatBounds);
        j = fallback;
    }
    return j;
}

__device__ __forceinline__ int32_t cell_index(const Args& A, int64_t p, int64_t c1) {
    if (p >= c1) return -1;
    int32_t cc = A.C[p];
    if (cc < 0 || cc >= A.nn) {
        atomicOr(A.status, kStatBounds);
        cc = 0;
    }
    return cc;
}

template <int ORDER>
__device__ __forceinline__ void put_cell(Smem32& S, int u, bool real, const float (&oh)[3], const float (&ol)[3]) {
    float v[10];
    if (real) {
        const float4 r0 = S.raw.c[u][0], r1 = S.raw.c[u][1], r2v = S.raw.c[u][2];
        v[0] = rel(r0.x, r1.x, oh[0], ol[0]);
        v[1] = rel(r0.y, r1.y, oh[1], ol[1]);
        v[2] = rel(r0.z, r1.z, oh[2], ol[2]);
        v[3] = r0.w;
        if (ORDER >= 2) {  // stored negated; Qzz = -(Qxx + Qyy)
            v[4] = -r1.w;
            v[5] = -r2v.x;
            v[6] = -r2v.y;
            v[7] = -r2v.z;
            v[8] = -r2v.w;
            v[9] = r1.w + r2v.z;
        }
    } else {  // padding entry: far away, massless
        v[0] = v[1] = v[2] = 1e15f;
        v[3] = 0.f;
#pragma unroll
        for (int a = 4; a < 10; ++a) v[a] = 0.f;
    }
    float* base = reinterpret_cast<float*>(&S.t.cp[u >> 1]);
    const int hh = u & 1;
#pragma unroll
    for (int a = 0; a < (ORDER >= 2 ? 10 : 4); ++a) base[2 * a + hh] = v[a];
}

// ---- tile loops --------------------------------------------------------------
// The hot loops note, per lane and without branching, which list pairs of
// the tile had a contact candidate (bit q of a mask); one reduction over the
// warp after the loop gives the pairs whose candidates are queued.
static_assert(kTileJ / 2 <= 32, "one mask bit per list pair of a tile");
template <int MODE, int R, bool TAIL, bool SELF>
__device__ __forceinline__ void pp_tile(const Args& A, Smem32& S, Chunk<R, TAIL>& K, int npair, int J, int tj,
                                        int& qn, int lane) {
    if constexpr (R > 0) {
        uint32_t hit = 0;
#pragma unroll kUnrollPP
        for (int q = 0; q < npair; ++q) {
            const JPair P = S.t.p.jp[q];
            const uint32_t* jid = &S.t.p.jid[2 * q];
            bool any = false;
#pragma unroll
            for (int r = 0; r < R; ++r) any |= pp_body<MODE, SELF>(A, P, jid, K.iv[r], K.nh[r], K.nl[r], K.g[r]);
            if (has_contact(MODE)) hit |= (uint32_t)any << q;
        }
        if (has_contact(MODE)) {
            uint32_t all = __reduce_or_sync(0xffffffffu, hit);
#pragma unroll 1
            while (all) {
                const int q = __ffs(all) - 1;
                all &= all - 1u;
                queue_pair<SELF, R, TAIL>(A, S, qn, S.t.p.jp[q], &S.t.p.jid[2 * q], K, 0, R, false, lane);
                if (qn >= 32) flush_queue(A, S, qn, lane);
            }
        }
    }
    if constexpr (TAIL) {
        const int trips = (npair + J - 1) / J;
        uint32_t hit = 0;
#pragma unroll 1
        for (int u = 0; u < trips; ++u) {
            const int q = u * J + tj;
            bool any = false;
            if (q < npair)
                any = pp_body<MODE, SELF>(A, S.t.p.jp[q], &S.t.p.jid[2 * q], K.iv[R], K.nh[R], K.nl[R], K.g[R]);
            if (has_contact(MODE)) hit |= (uint32_t)any << u;
        }
        if (has_contact(MODE)) {
            uint32_t all = __reduce_or_sync(0xffffffffu, hit);
#pragma unroll 1
            while (all) {
                const int u = __ffs(all) - 1;
                all &= all - 1u;
                const int q = u * J + tj;
                const bool ok = q < npair;
                queue_pair<SELF, R, TAIL>(A, S, qn, S.t.p.jp[ok ? q : 0], &S.t.p.jid[ok ? 2 * q : 0], K, R, R + 1, ok,
                                          lane);
                if (qn >= 32) flush_queue(A, S, qn, lane);
            }
        }
    }
}

template <int R, bool TAIL>
__device__ __forceinline__ void pp_far_tile(const Args& A, Smem32& S, Chunk<R, TAIL>& K, int npair, int J, int tj) {
    const float2 eps2 = f2(A.fp.eps2f);
    if constexpr (R > 0)
#pragma unroll kUnrollPP
        for (int q = 0; q < npair; ++q) {
            const JPair& P = S.t.p.jp[q];
#pragma unroll
            for (int r = 0; r < R; ++r) pp_far_body(P, K.nh[r], K.g[r], eps2);
        }
    if constexpr (TAIL)
#pragma unroll 1
        for (int q = tj; q < npair; q += J) pp_far_body(S.t.p.jp[q], K.nh[R], K.g[R], eps2);
}

template <int R, bool TAIL, int ORDER>
__device__ __forceinline__ void pc_tile(const Args& A, Smem32& S, Chunk<R, TAIL>& K, int npair, int J, int tj) {
    const float2 eps2 = f2(A.fp.eps2f);
    if constexpr (R > 0)
#pragma unroll kUnrollPC
        for (int q = 0; q < npair; ++q) {
            const CPair& Cp = S.t.cp[q];
#pragma unroll
            for (int r = 0; r < R; ++r) pc_body<ORDER>(Cp, K.nh[r], K.g[r], eps2);
        }
    if constexpr (TAIL)
#pragma unroll 1
        for (int q = tj; q < npair; q += J) pc_body<ORDER>(S.t.cp[q], K.nh[R], K.g[R], eps2);
}

template <int MODE, int R, bool TAIL, int ORDER>
__device__ __forceinline__ void group_chunk(const Args& A, Smem32& S, int64_t k, uint32_t b, uint32_t e,
                                            uint32_t i0, uint32_t ce, int T, const float (&oh)[3],
                                            const float (&ol)[3], int lane) {
    // group particles [b, e); this chunk's i-particles [i0, ce)
    constexpr int NS = Chunk<R, TAIL>::NS;
    Chunk<R, TAIL> K;
    const int J = TAIL ? 32 / T : 1;
    const int ti = TAIL ? lane % T : 0, tj = TAIL ? lane / T : 0;
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        const bool tail = (r == R);
        const uint32_t i = tail ? i0 + 32 * R + ti : i0 + 32 * r + lane;
        K.vl[r] = i < ce;
        K.iv[r] = K.vl[r] ? i : b;
        const float4 h = A.phi[K.iv[r]], l = A.plo[K.iv[r]];
        const float hv[3] = {h.x, h.y, h.z}, lv[3] = {l.x, l.y, l.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float rh, rl;
            rel2(hv[c], lv[c], oh[c], ol[c], rh, rl);
            K.nh[r][c] = f2(-rh);
            K.nl[r][c] = f2(-rl);
            K.g[r][c] = make_float2(0.f, 0.f);
            S.acc[32 * r + lane][c] = make_float2(0.f, 0.f);
        }
        S.abnd[32 * r + lane] = 0.f;
        S.hasc[32 * r + lane] = 0;
    }
    int qn = 0;
    __syncwarp();

    constexpr int PJ = kTileJ / 32, PC = kTileC / 32;  // staged entries per lane
    // (1) the group's own particles (contiguous), i = j excluded
    {
#pragma unroll
        for (int s = 0; s < PJ; ++s) {
            const uint32_t jj = b + lane + 32 * s;
            gather_particle(A, S, lane + 32 * s, jj < e ? jj : kNone);
        }
        cp_async_commit();
        for (uint32_t t0 = b; t0 < e; t0 += kTileJ) {
            const int nt = (int)min((uint32_t)kTileJ, e - t0);
            const int npair = (nt + 1) >> 1;
            cp_async_wait_all();
            __syncwarp();
#pragma unroll
            for (int s = 0; s < PJ; ++s) {
                const int u = lane + 32 * s;
                if (u < 2 * npair) put_particle<false>(S, u, u < nt, oh, ol);
            }
            __syncwarp();
#pragma unroll
            for (int s = 0; s < PJ; ++s) {
                const uint32_t jj = t0 + kTileJ + lane + 32 * s;
                gather_particle(A, S, lane + 32 * s, jj < e ? jj : kNone);
            }
            cp_async_commit();
            pp_tile<MODE, R, TAIL, true>(A, S, K, npair, J, tj, qn, lane);
            fold_all<R, TAIL>(S, K, lane);
            __syncwarp();
        }
        cp_async_wait_all();
        __syncwarp();
    }
    // (2) the other list particles: data gathered one tile ahead, indices two
    {
        const int64_t j0 = A.jj_off[k], j1 = A.jj_off[k + 1];
        const int64_t jm = A.jj_mid ? A.jj_mid[k] : j1;  // tiles from jm on are far
        uint32_t ib[PJ];
#pragma unroll
        for (int s = 0; s < PJ; ++s) {
            gather_particle(A, S, lane + 32 * s, list_index(A, j0 + lane + 32 * s, j1, b));
            ib[s] = list_index(A, j0 + kTileJ + lane + 32 * s, j1, b);
        }
        cp_async_commit();
        for (int64_t t0 = j0; t0 < j1; t0 += kTileJ) {
            const int nt = (int)min((int64_t)kTileJ, j1 - t0);
            const int npair = (nt + 1) >> 1;
            const bool far = t0 >= jm;
            cp_async_wait_all();
            __syncwarp();
#pragma unroll
            for (int s = 0; s < PJ; ++s) {
                const int u = lane + 32 * s;
                if (u < 2 * npair) {
                    if (far)
                        put_particle<true>(S, u, u < nt, oh, ol);
                    else
                        put_particle<false>(S, u, u < nt, oh, ol);
                }
            }
            __syncwarp();
#pragma unroll
            for (int s = 0; s < PJ; ++s) {
                gather_particle(A, S, lane + 32 * s, ib[s]);
                ib[s] = list_index(A, t0 + 2 * kTileJ + lane + 32 * s, j1, b);
            }
            cp_async_commit();
            if (far)
                pp_far_tile<R, TAIL>(A, S, K, npair, J, tj);
            else
                pp_tile<MODE, R, TAIL, false>(A, S, K, npair, J, tj, qn, lane);
            fold_all<R, TAIL>(S, K, lane);
            __syncwarp();
        }
        cp_async_wait_all();
        __syncwarp();
    }
    if (has_contact(MODE) && qn > 0) flush_queue(A, S, qn, lane);
    // (3) list cells: data gathered one tile ahead, indices two
    {
        const int64_t c0 = A.pc_off[k], c1 = A.pc_off[k + 1];
        int32_t cb[PC];
#pragma unroll
        for (int s = 0; s < PC; ++s) {
            gather_cell(A, S, lane + 32 * s, cell_index(A, c0 + lane + 32 * s, c1), ORDER >= 2 ? 3 : 2);
            cb[s] = cell_index(A, c0 + kTileC + lane + 32 * s, c1);
        }
        cp_async_commit();
        for (int64_t t0 = c0; t0 < c1; t0 += kTileC) {
            const int nt = (int)min((int64_t)kTileC, c1 - t0);
            const int npair = (nt + 1) >> 1;
            cp_async_wait_all();
            __syncwarp();
#pragma unroll
            for (int s = 0; s < PC; ++s) {
                const int u = lane + 32 * s;
                if (u < 2 * npair) put_cell<ORDER>(S, u, u < nt, oh, ol);
            }
            __syncwarp();
#pragma unroll
            for (int s = 0; s < PC; ++s) {
                gather_cell(A, S, lane + 32 * s, cb[s], ORDER >= 2 ? 3 : 2);
                cb[s] = cell_index(A, t0 + 2 * kTileC + lane + 32 * s, c1);
            }
            cp_async_commit();
            pc_tile<R, TAIL, ORDER>(A, S, K, npair, J, tj);
            fold_all<R, TAIL>(S, K, lane);
            __syncwarp();
        }
        cp_async_wait_all();
        __syncwarp();
    }
    __syncwarp();
    // (4) outputs: full slots directly, the tail slot after a reduction over its J lanes
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        const bool tail = (r == R);
        const int s = 32 * r + lane;
        double a[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] = A.fp.G * ((double)S.acc[s][c].x + (double)S.acc[s][c].y);
        float bnd = S.abnd[s];
        int hc = S.hasc[s];
        if (tail)
            for (int o = T; o < 32; o <<= 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
                bnd += __shfl_xor_sync(0xffffffffu, bnd, o);
                hc |= __shfl_xor_sync(0xffffffffu, hc, o);
            }
        if (K.vl[r] && (!tail || tj == 0)) {
            const uint32_t i = K.iv[r];
            // an ill-conditioned sum (terms far larger than the total) goes to
            // the refinement pass, which rewrites a_i
            const double kg = A.kref * A.fp.G;
            if (A.refine && hc) {  // judged with its contact term, after the contact pass
                A.cbnd[i] = bnd;
                A.cslot[i] = (uint32_t)k;
                A.cflag[i] = 1u;
            } else if (A.refine && a[0] * a[0] + a[1] * a[1] + a[2] * a[2] < kg * kg * (double)bnd) {
                const unsigned long long q = atomicAdd(A.nrefine, 1ull);
                A.refine[q] = make_uint2(i, (uint32_t)k);
            }
            if (A.add_central) central_newton(A.fp.GMc, A.x[i], A.y[i], A.z[i], a);
            A.ax[i] = a[0];
            A.ay[i] = a[1];
            A.az[i] = a[2];
        }
    }
    __syncwarp();
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// One group (list slot) for one warp.
template <int ORDER, int MODE>
__device__ __forceinline__ void force_group(const Args& A, Smem32& S, int64_t slot, int lane) {
    const int64_t k = A.order ? A.order[slot] : slot;  // groups of one size class run side by side
    const int32_t g = A.groups[k];
    const uint32_t b = A.begin[g], e = A.end[g];
    // origin: the group node's centre of mass as an FP32 hi/lo pair
    const float4 o0 = A.cell32[3 * (int64_t)g], o1 = A.cell32[3 * (int64_t)g + 1];
    const float oh[3] = {o0.x, o0.y, o0.z}, ol[3] = {o1.x, o1.y, o1.z};
    // chunks of at most A.chunk particles: R full slots plus a tail of at most 16
    for (uint32_t i0 = b; i0 < e;) {
        const uint32_t rem = e - i0, cnt = min(rem, (uint32_t)A.chunk);
        int R = (int)(cnt >> 5), t = (int)(cnt & 31), T = 0;
        if (t > 16) {
            ++R;  // more than half a slot left: a full one
        } else if (t > 0) {
            T = 1;
            while (T < t) T <<= 1;
        }
        const uint32_t ce = i0 + cnt;
        if (T > 0) {
            switch (R) {
                case 0: group_chunk<MODE, 0, true, ORDER>(A, S, k, b, e, i0, ce, T, oh, ol, lane); break;
                case 1: group_chunk<MODE, 1, true, ORDER>(A, S, k, b, e, i0, ce, T, oh, ol, lane); break;
                default: group_chunk<MODE, 2, true, ORDER>(A, S, k, b, e, i0, ce, T, oh, ol, lane); break;
            }
        } else {
            switch (R) {
                case 1: group_chunk<MODE, 1, false, ORDER>(A, S, k, b, e, i0, ce, 0, oh, ol, lane); break;
                case 2: group_chunk<MODE, 2, false, ORDER>(A, S, k, b, e, i0, ce, 0, oh, ol, lane); break;
                default: group_chunk<MODE, BH_F32_MAXR, false, ORDER>(A, S, k, b, e, i0, ce, 0, oh, ol, lane); break;
            }
        }
        i0 += cnt;
    }
}

// Warps per block = blockDim.x / 32 (at most BH_F32_MAXW); one Smem32 per warp.
template <int ORDER, int MODE>
__global__ void __launch_bounds__(32 * BH_F32_MAXW, 2) k_force32(const Args A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem32* sm = reinterpret_cast<Smem32*>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t wid = (int64_t)blockIdx.x * nw + w;
    Smem32& S = sm[w];
    const unsigned long long t0 = A.warp_time ? global_ns() : 0ull;
    if (A.abort && *A.abort) return;  // that build outgrew its buffers: the step is finished eagerly
    const int64_t ng = A.dng ? min(A.ng, (int64_t)*A.dng) : A.ng;
    if (A.ticket) {  // persistent, dynamic: the next list slot from the shared counter
        for (;;) {
            unsigned long long s = 0;
            if (lane == 0) s = atomicAdd(A.ticket, 1ull);
            s = __shfl_sync(0xffffffffu, s, 0);
            if ((int64_t)s >= ng) break;
            force_group<ORDER, MODE>(A, S, (int64_t)s, lane);
        }
    } else {  // static: one slot per warp (grid) or every stride-th slot (persistent)
        const int64_t stride = (int64_t)gridDim.x * nw;
        for (int64_t s = wid; s < ng; s += stride) force_group<ORDER, MODE>(A, S, s, lane);
    }
    if (A.warp_time && lane == 0) {
        A.warp_time[2 * wid] = t0;
        A.warp_time[2 * wid + 1] = global_ns();
    }
}

// Size class of a group = the (R, tail) variant of its last chunk; classes
// are numbered so that larger work comes first.
__device__ __forceinline__ int size_class(uint32_t n_i, uint32_t chunk) {
    const uint32_t rem = n_i - chunk * ((n_i - 1u) / chunk);
    int R = (int)(rem >> 5);
    const int t = (int)(rem & 31);
    bool tail = false;
    if (t > 16)
        ++R;
    else if (t > 0)
        tail = true;
    const int cls = 2 * R + (tail ? 1 : 0) - 1;  // (0,T)=0 (1,F)=1 (1,T)=2 (2,F)=3 (2,T)=4 (3,F)=5
    return 5 - cls;
}

// Processing order: size class first (warps side by side run the same code),
// then, with cost ordering on, largest estimated cost first within a class
// (cost = n_i (n_i + list particles + 2 list cells), bucketed by log2), so the
// list ends with the cheapest groups of each class.
constexpr int kCostBuckets = 32;
constexpr int kOrderBuckets = 6 * kCostBuckets;

__device__ __forceinline__ int order_bucket(int64_t k, const int32_t* __restrict__ groups,
                                            const uint32_t* __restrict__ begin, const uint32_t* __restrict__ end,
                                            const int64_t* __restrict__ jj_off, const int64_t* __restrict__ pc_off,
                                            uint32_t chunk, bool by_cost) {
    const int32_t g = groups[k];
    const uint32_t ni = end[g] - begin[g];
    int cb = 0;
    if (by_cost) {
        const unsigned long long cost =
            (unsigned long long)ni * ((unsigned long long)ni + (unsigned long long)(jj_off[k + 1] - jj_off[k]) +
                                      2ull * (unsigned long long)(pc_off[k + 1] - pc_off[k]));
        const int lg = cost ? 63 - __clzll((long long)cost) : 0;
        cb = kCostBuckets - 1 - min(lg, kCostBuckets - 1);
    }
    return size_class(ni, chunk) * kCostBuckets + cb;
}

__global__ void k_order_hist(int64_t ng, const unsigned long long* __restrict__ dng,
                             const int32_t* __restrict__ groups, const uint32_t* __restrict__ begin,
                             const uint32_t* __restrict__ end, const int64_t* __restrict__ jj_off,
                             const int64_t* __restrict__ pc_off, uint32_t chunk, bool by_cost,
                             unsigned long long* cnt) {
    if (dng) ng = min(ng, (int64_t)*dng);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[order_bucket(k, groups, begin, end, jj_off, pc_off, chunk, by_cost)], 1ull);
}

// Windowed order: key = (group index / window, bucket); a stable sort of the
// keys keeps list (Morton) order within a window and a bucket, so the warps
// running at one time work on one stretch of the ring (their list data
// overlaps in L2) while the warps side by side still share a size class.
__global__ void k_order_keys(int64_t ng, const int32_t* __restrict__ groups, const uint32_t* __restrict__ begin,
                             const uint32_t* __restrict__ end, const int64_t* __restrict__ jj_off,
                             const int64_t* __restrict__ pc_off, uint32_t chunk, bool by_cost, int64_t window,
                             uint64_t* __restrict__ keys) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    keys[k] = ((uint64_t)(k / window) << 8) | (uint64_t)order_bucket(k, groups, begin, end, jj_off, pc_off, chunk, by_cost);
}

// exclusive prefix of the bucket counts (one block of kOrderBuckets threads)
__global__ void k_order_prefix(unsigned long long* cnt) {
    __shared__ unsigned long long v[kOrderBuckets];
    v[threadIdx.x] = cnt[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int b = 0; b < kOrderBuckets; ++b) {
            const unsigned long long t = v[b];
            v[b] = run;
            run += t;
        }
    }
    __syncthreads();
    cnt[threadIdx.x] = v[threadIdx.x];
}

__global__ void k_order_scatter(int64_t ng, const unsigned long long* __restrict__ dng,
                                const int32_t* __restrict__ groups, const uint32_t* __restrict__ begin,
                                const uint32_t* __restrict__ end, const int64_t* __restrict__ jj_off,
                                const int64_t* __restrict__ pc_off, uint32_t chunk, bool by_cost,
                                const unsigned long long* __restrict__ start, unsigned long long* cursor,
                                int32_t* __restrict__ order) {
    if (dng) ng = min(ng, (int64_t)*dng);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += (int64_t)gridDim.x * blockDim.x) {
        const int b = order_bucket(k, groups, begin, end, jj_off, pc_off, chunk, by_cost);
        order[start[b] + atomicAdd(&cursor[b], 1ull)] = (int32_t)k;
    }
}

// FP64 pass over the contact candidates: Eq. (1) in the oracle's operation
// order less the gravity the FP32 kernel already added for the pair (r_coll
// or r clamp), i.e. the spring and dashpot term when r <= r_coll.
//
// The candidates arrive in no fixed order (warps append them as they go), so
// the terms are summed per particle in 64-bit fixed point (units of 2^-50,
// terms below 2^10 in magnitude): integer addition does not depend on the
// order, which keeps every run bit-reproducible.  Three passes: clear the
// accumulators of the particles involved, add the terms, then move each
// particle's sum into its acceleration (the first pass to take it adds the
// whole sum, every later one adds zero).
constexpr double kFix = 1125899906842624.0;  // 2^50
constexpr double kFixMax = 1024.0;

__device__ __forceinline__ int64_t contact_count(const unsigned long long* count, int64_t cap, int* status,
                                                 bool flag) {
    int64_t np = (int64_t)*count;
    if (np > cap) {
        np = cap;
        if (flag && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatListOverflow);
    }
    return np;
}

__global__ void k_contacts_clear(const uint2* __restrict__ pairs, const unsigned long long* __restrict__ count,
                                 int64_t cap, unsigned long long* __restrict__ acc, int* status) {
    const int64_t np = contact_count(count, cap, status, true);
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < np; u += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = pairs[u].x;
        acc[3 * (int64_t)i] = acc[3 * (int64_t)i + 1] = acc[3 * (int64_t)i + 2] = 0ull;
    }
}

__global__ void k_contacts64(const uint2* __restrict__ pairs, const unsigned long long* __restrict__ count,
                             int64_t cap, ForceParams fp, const double* __restrict__ x,
                             const double* __restrict__ y, const double* __restrict__ z,
                             const double* __restrict__ vx, const double* __restrict__ vy,
                             const double* __restrict__ vz, const double* __restrict__ m,
                             unsigned long long* __restrict__ acc, unsigned long long* n_touch, int* status) {
    const int64_t np = contact_count(count, cap, status, false);
    unsigned long long touching = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < np; u += (int64_t)gridDim.x * blockDim.x) {
        const uint2 pr = pairs[u];
        const uint32_t i = pr.x, j = pr.y;
        double a[3] = {0.0, 0.0, 0.0};
        touching += contact_term64(fp, x[i], y[i], z[i], vx[i], vy[i], vz[i], m[i], x[j], y[j], z[j], vx[j], vy[j],
                                   vz[j], m[j], a);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double v = a[c];
            if (!(fabs(v) < kFixMax)) {  // outside the fixed-point range (or not finite)
                atomicOr(status, kStatRange);
                v = 0.0;
            }
            atomicAdd(&acc[3 * (int64_t)i + c], (unsigned long long)__double2ll_rn(v * kFix));
        }
    }
    if (touching) atomicAdd(n_touch, touching);
}

__global__ void k_contacts_apply(const uint2* __restrict__ pairs, const unsigned long long* __restrict__ count,
                                 int64_t cap, unsigned long long* __restrict__ acc, double* ax, double* ay,
                                 double* az, int* status) {
    const int64_t np = contact_count(count, cap, status, false);
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < np; u += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = pairs[u].x;
        double* out[3] = {ax, ay, az};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long v = (long long)atomicExch(&acc[3 * (int64_t)i + c], 0ull);
            if (v != 0) atomicAdd(&out[c][i], (double)v / kFix);
        }
    }
}

// ---- refinement of ill-conditioned particles ------------------------------
// A particle whose FP32 sum is ill-conditioned (|a_i| small against the sum
// of |tile partial sums|, e.g. where the pull of its neighbours nearly
// cancels) is evaluated again, over the same group lists and in the same
// terms (Eq. (1)'s gravity with the r_coll floor; monopole + quadrupole),
// in df arithmetic (hi + lo pairs of FP32 numbers, about 44 bits; see
// dfloat.cuh) from the hi/lo particle coordinates and masses and the cell
// records with their mass corrections, with the contact terms of its pairs
// within reach evaluated in FP64 as the contact pass does.  One warp per
// queued particle; the lanes split the entries and the partial sums are
// reduced in df.  The result replaces a_i; the pass runs after the contact
// pass, whose terms it includes.  A particle with a contact candidate is
// judged only after that pass (k_flag_contacts): the spring term can cancel
// the pull of the neighbour it touches.
struct RefineConsts {
    df rc2, eps2, rc2eps2;  // r_coll^2, eps^2, r_coll^2 + eps^2
};

__device__ __forceinline__ df df_of(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ void ref_pp(const Args& A, const RefineConsts& K, float xh, float xl, float yh, float yl,
                                       float zh, float zl, uint32_t i, uint32_t j, const float4 h, const float4 l,
                                       df (&acc)[3], double (&ac)[3]) {
    const df d[3] = {df_diff(h.x, l.x, xh, xl), df_diff(h.y, l.y, yh, yl), df_diff(h.z, l.z, zh, zl)};
    const df r2 = df_dot3(d[0], d[1], d[2]);
    if (r2.hi == 0.f) return;  // coincident pair: no term
    if (r2.hi < A.rc2chk)  // the contact term of the FP64 pass, decided and evaluated as there
        contact_term64(A.fp, A.x[i], A.y[i], A.z[i], A.vx[i], A.vy[i], A.vz[i], A.m[i], A.x[j], A.y[j], A.z[j],
                       A.vx[j], A.vy[j], A.vz[j], A.m[j], ac);
    const df s2 = df_gt(r2, K.rc2) ? df_add(r2, K.eps2) : K.rc2eps2;
    const df y = df_rsqrt(s2);
    const df f = df_mul(df_mul(fast_two_sum(h.w, l.w), y), df_mul(y, y));  // m / s^3
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = df_add(acc[c], df_mul(f, d[c]));
}

struct CellRec {
    float4 r0, r1, r2;
    float mlo;
};

__device__ __forceinline__ CellRec load_cell(const Args& A, const float* __restrict__ mlo, int32_t cc) {
    return {A.cell32[3 * (int64_t)cc], A.cell32[3 * (int64_t)cc + 1], A.cell32[3 * (int64_t)cc + 2], mlo[cc]};
}

__device__ __forceinline__ void ref_pc(const Args& A, const RefineConsts& K, float xh, float xl, float yh, float yl,
                                       float zh, float zl, const CellRec& cr, df (&acc)[3]) {
    const float4 r0 = cr.r0, r1 = cr.r1;
    // R = x_i - c (the oracle's sign); a = -M R / R^3 + Q R / R^5 - 5/2 (R.Q.R) R / R^7 (G-free)
    const df R[3] = {df_diff(xh, xl, r0.x, r1.x), df_diff(yh, yl, r0.y, r1.y), df_diff(zh, zl, r0.z, r1.z)};
    const df R2 = df_add(df_dot3(R[0], R[1], R[2]), K.eps2);
    const df y = df_rsqrt(R2);
    const df y2 = df_mul(y, y);
    const df y3 = df_mul(y2, y);
    const df M = fast_two_sum(r0.w, cr.mlo);
    const df mono = df_neg(df_mul(M, y3));
    df t[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) t[c] = df_mul(mono, R[c]);
    if (A.fp.order >= 2) {
        // the quadrupole part, at most about theta^2 of the monopole, in FP32
        // from the df separation (its FP32 rounding stays far below the
        // monopole's df accuracy)
        const float4 r2v = cr.r2;
        const float qxx = r1.w, qxy = r2v.x, qxz = r2v.y, qyy = r2v.z, qyz = r2v.w, qzz = -(qxx + qyy);
        const float Rx = R[0].hi, Ry = R[1].hi, Rz = R[2].hi;
        const float qx = qxx * Rx + qxy * Ry + qxz * Rz, qy = qxy * Rx + qyy * Ry + qyz * Rz,
                    qz = qxz * Rx + qyz * Ry + qzz * Rz;
        const float rqr = Rx * qx + Ry * qy + Rz * qz;
        const float yf = y.hi, y2f = yf * yf, y5f = y2f * y2f * yf;
        const float w = -2.5f * rqr * y5f * y2f;  // -5/2 (R.Q.R) / R^7
        t[0] = df_add(t[0], df_make(y5f * qx + w * Rx));
        t[1] = df_add(t[1], df_make(y5f * qy + w * Ry));
        t[2] = df_add(t[2], df_make(y5f * qz + w * Rz));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = df_add(acc[c], t[c]);
}

// After the contact pass: each particle with a contact candidate (claimed
// once through its flag) is queued when its tree part, gravity and contact,
// is small against its FP32 bound.
__global__ void k_flag_contacts(const Args A, const uint2* __restrict__ pairs, const unsigned long long* count,
                                int64_t cap) {
    int64_t np = (int64_t)*count;
    if (np > cap) np = cap;
    const double kg = A.kref * A.fp.G;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < np; u += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = pairs[u].x;
        if (i >= A.n || atomicExch(&A.cflag[i], 0u) == 0u) continue;
        double a[3] = {A.ax[i], A.ay[i], A.az[i]};
        if (A.add_central) {  // the tree part: the central term taken off again
            double c[3] = {0.0, 0.0, 0.0};
            central_newton(A.fp.GMc, A.x[i], A.y[i], A.z[i], c);
#pragma unroll
            for (int q = 0; q < 3; ++q) a[q] -= c[q];
        }
        if (a[0] * a[0] + a[1] * a[1] + a[2] * a[2] < kg * kg * (double)A.cbnd[i]) {
            const unsigned long long q = atomicAdd(A.nrefine, 1ull);
            if ((int64_t)q < (int64_t)A.n) A.refine[q] = make_uint2(i, A.cslot[i]);
        }
    }
}

// Launch bounds for 4 blocks of 8 warps per SM (64 registers, a few small
// spills): the df chains are latency-bound, and 32 warps per SM refine a
// 2^26 ring in 6.1 ms against 6.6 ms at 16 warps (97 registers).
__global__ void __launch_bounds__(256, 4) k_refine32(const Args A, const RefineConsts K,
                                                     const float* __restrict__ mlo, int64_t cap) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t cnt = (int64_t)*A.nrefine;
    if (cnt > cap) cnt = cap;  // cannot happen: one entry per particle at most
    for (int64_t q = wid; q < cnt; q += nw) {
        const uint2 e = A.refine[q];
        const uint32_t i = e.x;
        const int64_t k = e.y;
        if (i >= A.n || k >= A.ng) {
            if (lane == 0) atomicOr(A.status, kStatBounds);
            continue;
        }
        const int32_t g = A.groups[k];
        const uint32_t b = A.begin[g], en = A.end[g];
        const float4 hi = A.phi[i], lo = A.plo[i];
        df acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        double ac[3] = {0.0, 0.0, 0.0};  // contact terms (FP64)
        // each loop loads the next entry's data before evaluating the current one
        {
            uint32_t j = b + lane;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (j < en) {
                h = A.phi[j];
                l = A.plo[j];
            }
            for (; j < en; j += 32) {
                const uint32_t jn = j + 32;
                float4 hn = h, ln = l;
                if (jn < en) {
                    hn = A.phi[jn];
                    ln = A.plo[jn];
                }
                if (j != i) ref_pp(A, K, hi.x, lo.x, hi.y, lo.y, hi.z, lo.z, i, j, h, l, acc, ac);
                h = hn;
                l = ln;
            }
        }
        {
            const int64_t j1 = A.jj_off[k + 1];
            int64_t p = A.jj_off[k] + lane;
            auto index = [&](int64_t q) -> uint32_t {
                if (q >= j1) return kNone;
                const uint32_t j = A.JJ[q];
                if (j >= A.n) {
                    atomicOr(A.status, kStatBounds);
                    return kNone;
                }
                return j;
            };
            uint32_t j = index(p), jn = index(p + 32);
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (j != kNone) {
                h = A.phi[j];
                l = A.plo[j];
            }
            for (; p < j1; p += 32) {
                const uint32_t jnn = index(p + 64);
                float4 hn = h, ln = l;
                if (jn != kNone) {
                    hn = A.phi[jn];
                    ln = A.plo[jn];
                }
                if (j != kNone) ref_pp(A, K, hi.x, lo.x, hi.y, lo.y, hi.z, lo.z, i, j, h, l, acc, ac);
                j = jn;
                jn = jnn;
                h = hn;
                l = ln;
            }
        }
        {
            const int64_t c1 = A.pc_off[k + 1];
            int64_t p = A.pc_off[k] + lane;
            auto index = [&](int64_t q) -> int32_t {
                if (q >= c1) return -1;
                const int32_t cc = A.C[q];
                if (cc < 0 || cc >= A.nn) {
                    atomicOr(A.status, kStatBounds);
                    return -1;
                }
                return cc;
            };
            int32_t cc = index(p), cn = index(p + 32);
            CellRec cr = {};
            if (cc >= 0) cr = load_cell(A, mlo, cc);
            for (; p < c1; p += 32) {
                const int32_t cnn = index(p + 64);
                CellRec crn = cr;
                if (cn >= 0) crn = load_cell(A, mlo, cn);
                if (cc >= 0) ref_pc(A, K, hi.x, lo.x, hi.y, lo.y, hi.z, lo.z, cr, acc);
                cc = cn;
                cn = cnn;
                cr = crn;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const df v = {__shfl_xor_sync(0xffffffffu, acc[c].hi, o), __shfl_xor_sync(0xffffffffu, acc[c].lo, o)};
                acc[c] = df_add(acc[c], v);
                ac[c] += __shfl_xor_sync(0xffffffffu, ac[c], o);
            }
        if (lane == 0) {
            double a[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) a[c] = A.fp.G * df_to_double(acc[c]) + ac[c];
            if (A.add_central) central_newton(A.fp.GMc, A.x[i], A.y[i], A.z[i], a);
            A.ax[i] = a[0];
            A.ay[i] = a[1];
            A.az[i] = a[2];
        }
    }
}

using Force32Fn = void (*)(const Args);

Force32Fn force32_kernel(int order, int mode) {
    if (order >= 2) {
        switch (mode) {
            case kContact: return k_force32<2, kContact>;
            case kPlain: return k_force32<2, kPlain>;
            case kMask: return k_force32<2, kMask>;
            default: return k_force32<2, kContact0>;
        }
    }
    switch (mode) {
        case kContact: return k_force32<1, kContact>;
        case kPlain: return k_force32<1, kPlain>;
        case kMask: return k_force32<1, kMask>;
        default: return k_force32<1, kContact0>;
    }
}

int resident_blocks(Force32Fn kern, int warps) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * warps, warps * (int)sizeof(Smem32)) !=
        cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

}  // namespace

// Processing order of the groups for the FP32 kernel (once per list build).
int build_order32(Ctx* c) {
    const int64_t ng = c->n_groups;
    BH_TRY(grow(c, c->order, (size_t)ng + 1, "group order"));
    BH_TRY(grow(c, c->order_cnt, 2 * (size_t)kOrderBuckets, "group order buckets"));
    unsigned long long* cnt = c->order_cnt.p;
    const uint32_t chunk = (uint32_t)std::min(c->tune.chunk, 32 * BH_F32_MAXR);
    const bool by_cost = c->tune.order_by_cost != 0;
    if (c->tune.order_window > 0 && ng > c->tune.order_window && !c->dev_build) {  // (device-sized: plain order)
        for (int b = 0; b < 2; ++b) {
            BH_TRY(grow(c, c->ord_key[b], (size_t)ng, "group order keys"));
            BH_TRY(grow(c, c->ord_idx[b], (size_t)ng, "group order indices"));
        }
        BH_TRY(grow(c, c->ord_scratch, (size_t)sort_scratch_words(ng), "group order sort scratch"));
        k_order_keys<<<blocks_for(ng, 256), 256, 0, c->stream>>>(ng, c->groups.p, c->begin.p, c->end.p, c->cnt_j.p,
                                                                 c->cnt_c.p, chunk, by_cost, c->tune.order_window,
                                                                 c->ord_key[0].p);
        BH_LAUNCH(c);
        if (c->sort_attr_device != c->device) {
            BH_CUDA(c, sort_setup_device());
            c->sort_attr_device = c->device;
        }
        BH_CUDA(c, sort_pairs_with(c->stream, c->ord_key[0].p, c->ord_idx[0].p, c->ord_key[1].p, c->ord_idx[1].p, ng,
                                   c->ord_scratch.p));
        c->n_launches += 1 + 8 * 5;
        BH_CUDA(c, cudaMemcpyAsync(c->order.p, c->ord_idx[0].p, ng * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                   c->stream));
        return BH_OK;
    }
    // device-sized build: the group count is read on the device
    const unsigned long long* dng = c->dev_build ? c->d_sz + kSzNg : nullptr;
    const unsigned nb = dng ? (unsigned)(4 * c->num_sms) : blocks_for(ng, 256);
    BH_CUDA(c, cudaMemsetAsync(cnt, 0, 2 * kOrderBuckets * sizeof(unsigned long long), c->stream));
    k_order_hist<<<nb, 256, 0, c->stream>>>(ng, dng, c->groups.p, c->begin.p, c->end.p, c->cnt_j.p, c->cnt_c.p, chunk,
                                            by_cost, cnt);
    BH_LAUNCH(c);
    k_order_prefix<<<1, kOrderBuckets, 0, c->stream>>>(cnt);
    BH_LAUNCH(c);
    k_order_scatter<<<nb, 256, 0, c->stream>>>(ng, dng, c->groups.p, c->begin.p, c->end.p, c->cnt_j.p, c->cnt_c.p,
                                               chunk, by_cost, cnt, cnt + kOrderBuckets, c->order.p);
    BH_LAUNCH(c);
    return BH_OK;
}

namespace {
RefineConsts refine_consts(const ForceParams& fp) {
    auto split = [](double v) {
        const float h = (float)v;
        return df{h, (float)(v - (double)h)};
    };
    return RefineConsts{split(fp.rc2), split(fp.eps2), split(fp.rc2 + fp.eps2)};
}

// The refinement pass over the particles the force kernel queued (count
// read on the device, so it can run inside a captured graph).
int refine_pass(Ctx* c, const Args& A, const ForceParams& fp) {
    if (!A.refine) return BH_OK;
    BH_TRY(stage_begin(c, BH_STAGE_REFINE));
    k_refine32<<<(unsigned)(c->num_sms * 4), 256, 0, c->stream>>>(A, refine_consts(fp), c->cell32lo.p,
                                                                   (int64_t)c->refine.cap);
    BH_LAUNCH(c);
    return stage_end(c);
}

// The particles with contact candidates, judged after the contact pass.
int flag_pass(Ctx* c, const Args& A, unsigned nb) {
    if (!A.refine) return BH_OK;
    BH_TRY(stage_begin(c, BH_STAGE_REFINE));
    k_flag_contacts<<<nb, 128, 0, c->stream>>>(A, A.contacts, A.ncontact, A.contact_cap);
    BH_LAUNCH(c);
    return stage_end(c);
}

int contact_pass(Ctx* c, const Args& A, const ForceParams& fp, bh_particles* p, unsigned nb) {
    BH_TRY(stage_begin(c, BH_STAGE_CONTACTS));
    unsigned long long* acc = c->contact_acc.p;
    k_contacts_clear<<<nb, 128, 0, c->stream>>>(A.contacts, A.ncontact, A.contact_cap, acc, c->d_status);
    BH_LAUNCH(c);
    k_contacts64<<<nb, 128, 0, c->stream>>>(A.contacts, A.ncontact, A.contact_cap, fp, p->x, p->y, p->z, p->vx, p->vy,
                                            p->vz, p->m, acc, c->d_small + 18, c->d_status);
    BH_LAUNCH(c);
    k_contacts_apply<<<nb, 128, 0, c->stream>>>(A.contacts, A.ncontact, A.contact_cap, acc, p->ax, p->ay, p->az,
                                                c->d_status);
    BH_LAUNCH(c);
    return stage_end(c);
}
}  // namespace

int launch_force32(Ctx* c, bh_particles* p, const ForceParams& fp, bool add_central) {
    Args A;
    A.ng = c->n_groups;
    A.dng = c->dev_build ? c->d_sz + kSzNg : nullptr;
    A.abort = c->abort;
    A.order = c->order.p;
    A.groups = c->groups.p;
    A.begin = c->begin.p;
    A.end = c->end.p;
    A.jj_off = c->cnt_j.p;
    A.jj_mid = c->cnt_jm.p;
    A.JJ = c->JJ.p;
    A.pc_off = c->cnt_c.p;
    A.C = c->C.p;
    A.phi = c->phi.p;
    A.plo = c->plo.p;
    A.cell32 = c->cell32.p;
    A.x = p->x;
    A.y = p->y;
    A.z = p->z;
    A.ax = p->ax;
    A.ay = p->ay;
    A.az = p->az;
    const bool contact = c->prm.r_coll > 0.0;
    const int64_t cap = c->n > 65536 ? c->n : 65536;
    if (contact && c->contacts.cap < (size_t)cap) BH_TRY(grow(c, c->contacts, (size_t)cap, "contact pairs"));
    if (contact) BH_TRY(grow(c, c->contact_acc, 3 * (size_t)c->n, "contact sums"));
    A.contacts = reinterpret_cast<uint2*>(c->contacts.p);
    A.contact_cap = (int64_t)c->contacts.cap;
    if (c->capturing && c->tune.graph_contact_room > 0)  // the room a graph step may use
        A.contact_cap = std::min(A.contact_cap, (int64_t)c->tune.graph_contact_room);
    A.ncontact = c->d_small + 16;
    c->contact_stats = contact;
    BH_CUDA(c, cudaMemsetAsync(A.ncontact, 0, sizeof(unsigned long long), c->stream));
    BH_CUDA(c, cudaMemsetAsync(c->d_small + 18, 0, sizeof(unsigned long long), c->stream));  // pairs in contact
    A.n = (uint32_t)c->n;
    A.nn = c->n_nodes;
    A.status = c->d_status;
    A.fp = fp;
    A.floor2 = (float)(fp.rc2 + fp.eps2);
    A.rc2chk = (float)(fp.rc2 * (1.0 + 1e-5));
    A.add_central = add_central;
    const int mode = contact ? (fp.eps2f == 0.f ? kContact0 : kContact) : (A.floor2 > 0.f ? kPlain : kMask);
    const Force32Fn kern = force32_kernel(c->prm.order, mode);
    const int W = c->tune.warps;
    const int smem = (int)(W * sizeof(Smem32));
    if (c->f32_attr_device != c->device) {  // once per device: room for the largest block
        const int smax = (int)(BH_F32_MAXW * sizeof(Smem32));
        for (int o = 1; o <= 2; ++o)
            for (int m = 0; m < 4; ++m)
                BH_CUDA(c, cudaFuncSetAttribute(force32_kernel(o, m), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                smax));
        c->f32_attr_device = c->device;
    }
    A.chunk = std::min(c->tune.chunk, 32 * BH_F32_MAXR);
    A.ticket = nullptr;
    A.warp_time = nullptr;
    A.kref = BH_REFINE_K;
    A.nrefine = c->d_small + 20;
    A.refine = nullptr;
    A.cbnd = nullptr;
    A.cslot = nullptr;
    A.cflag = nullptr;
    A.vx = p->vx;
    A.vy = p->vy;
    A.vz = p->vz;
    A.m = p->m;
    if (A.kref > 0.0) {
        BH_TRY(grow(c, c->refine, (size_t)c->n, "refinement queue"));
        A.refine = c->refine.p;
        if (contact) {
            const bool fresh = c->cflag.cap < (size_t)c->n;
            BH_TRY(grow(c, c->cbnd, (size_t)c->n, "contact-particle bounds"));
            BH_TRY(grow(c, c->cslot, (size_t)c->n, "contact-particle list slots"));
            BH_TRY(grow(c, c->cflag, (size_t)c->n, "contact-particle flags"));
            if (fresh) BH_CUDA(c, cudaMemsetAsync(c->cflag.p, 0, c->cflag.cap * sizeof(unsigned), c->stream));
            A.cbnd = c->cbnd.p;
            A.cslot = c->cslot.p;
            A.cflag = c->cflag.p;
        }
    }
    unsigned nb;
    if (c->tune.sched == BH_SCHED_GRID && !A.dng) {
        nb = blocks_for(A.ng, W);
    } else {  // (a device-sized build runs the grid schedule as a persistent static one)
        nb = (unsigned)(c->num_sms * resident_blocks(kern, W));
        const int64_t need = (A.ng + W - 1) / W;
        if ((int64_t)nb > need) nb = (unsigned)(need > 0 ? need : 1);
        if (c->tune.sched == BH_SCHED_DYNAMIC) {
            A.ticket = c->d_small + 17;
            BH_CUDA(c, cudaMemsetAsync(A.ticket, 0, sizeof(unsigned long long), c->stream));
        }
        if (c->timing && !c->capturing) {
            BH_TRY(grow(c, c->warp_time, 2 * (size_t)nb * W, "warp times"));
            A.warp_time = c->warp_time.p;
            c->warp_time_n = (int64_t)nb * W;
        }
    }
    c->f32_blocks = nb;
    c->refine_pending = A.refine != nullptr;  // its count is read when asked for
    for (int attempt = 0; attempt < 2; ++attempt) {
        BH_CUDA(c, cudaMemsetAsync(A.nrefine, 0, sizeof(unsigned long long), c->stream));
        BH_TRY(timing_begin(c));
        BH_TRY(stage_begin(c, BH_STAGE_FORCE));
        kern<<<nb, 32 * W, smem, c->stream>>>(A);
        BH_LAUNCH(c);
        BH_TRY(stage_end(c));
        BH_TRY(timing_end(c));
        if (!contact) {
            BH_TRY(refine_pass(c, A, fp));
            break;
        }
        if (c->capturing) {
            // inside a captured graph: no read-back; the passes take the count
            // from the device and an overflow is flagged in the status word
            const unsigned nbc = (unsigned)(c->num_sms * 4);
            BH_TRY(contact_pass(c, A, fp, p, nbc));
            BH_TRY(flag_pass(c, A, nbc));
            BH_TRY(refine_pass(c, A, fp));
            break;
        }
        // size the FP64 contact pass (one read-back per evaluation); on
        // overflow grow the list and evaluate again
        unsigned long long np = 0;
        BH_CUDA(c, cudaMemcpyAsync(&np, A.ncontact, sizeof(np), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
        c->n_contacts = (int64_t)np;
        if ((int64_t)np > A.contact_cap) {
            BH_TRY(grow(c, c->contacts, (size_t)(np + np / 4 + 1024), "contact pairs"));
            A.contacts = reinterpret_cast<uint2*>(c->contacts.p);
            A.contact_cap = (int64_t)c->contacts.cap;
            BH_CUDA(c, cudaMemsetAsync(A.ncontact, 0, sizeof(unsigned long long), c->stream));
            if (A.ticket) BH_CUDA(c, cudaMemsetAsync(A.ticket, 0, sizeof(unsigned long long), c->stream));
            continue;
        }
        if (np > 0) {
            BH_TRY(contact_pass(c, A, fp, p, blocks_for((int64_t)np, 128)));
            BH_TRY(flag_pass(c, A, blocks_for((int64_t)np, 128)));
        }
        BH_TRY(refine_pass(c, A, fp));
        break;
    }
    return BH_OK;
}

}  // namespace bh
