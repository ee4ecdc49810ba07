// force.cu -- Sec. 4.2 step 3d, second half: the double loop over the
// particles of a group and the entries of its shared interaction list.
//
//   list particles: Eq. (1) read as an acceleration (gravity G m_j r/r^3,
//                   softened by eps, held at its r_coll value inside r_coll,
//                   plus the spring/dashpot contact term inside r_coll);
//   list cells:     centre-of-mass monopole (Sec. 5.1) and, for order 2, the
//                   traceless quadrupole about the centre of mass.
//
// Two kernels:
//   k_force64  plain FP64 (absolute coordinates).
//   k_force32  FP32 on coordinates relative to the group's FP64 centre of
//              mass (Sec. 4.7 shifts to "one of the particles which share the
//              list"; any point of the group bounds the shifted coordinates
//              the same way).  The shift uses a per-step hi/lo FP32 split of
//              every FP64 coordinate, (x_hi - o_hi) + (x_lo - o_lo), which is
//              within one FP32 rounding of the FP64-shifted value and keeps
//              FP64 arithmetic (1/64 of the FP32 rate on this GPU) out of the
//              inner loops.  Contact pairs are re-decided and evaluated in
//              FP64 in a rarely taken branch, so the r <= r_coll decision is
//              the FP64 one.
//
// Mapping: one warp per group; list entries are staged 32 at a time into the
// warp's shared-memory tile (gather + shift), then broadcast from shared
// memory to the lanes, each lane holding R i-particles in registers.
#include "bh_internal.cuh"

namespace bh {
namespace {

struct ForceParams {
    double G, eps2, rc2, rc2_hi, kappa, eta, r_coll, GMc;
    float eps2f, floor2f, rc2chk_f;
    int order;
};

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Exact (oracle-order, no contraction) evaluation of Eq. (1) for a pair that
// may be in contact; adds G-free gravity to *g and the contact term to *cn.
// Returns without effect for coincident positions.
__device__ __forceinline__ void near_pair64(const ForceParams& fp, double xi, double yi, double zi,
                                            double vxi, double vyi, double vzi, double mi, double xj,
                                            double yj, double zj, double vxj, double vyj, double vzj,
                                            double mj, double* g, double* cn) {
    const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (r2 == 0.0) return;
    if (r2 > fp.rc2) {
        const double s2 = __dadd_rn(r2, fp.eps2);
        const double f = __ddiv_rn(mj, __dmul_rn(s2, __dsqrt_rn(s2)));
        g[0] += f * dx;
        g[1] += f * dy;
        g[2] += f * dz;
        return;
    }
    const double s2 = __dadd_rn(fp.rc2, fp.eps2);
    const double fg = __ddiv_rn(mj, __dmul_rn(s2, __dsqrt_rn(s2)));
    g[0] += fg * dx;
    g[1] += fg * dy;
    g[2] += fg * dz;
    const double r = __dsqrt_rn(r2);
    const double dvx = __dsub_rn(vxj, vxi), dvy = __dsub_rn(vyj, vyi), dvz = __dsub_rn(vzj, vzi);
    const double rv = __dadd_rn(__dadd_rn(__dmul_rn(dx, dvx), __dmul_rn(dy, dvy)), __dmul_rn(dz, dvz));
    const double fc = __ddiv_rn(mj, __dadd_rn(mi, mj)) *
                      (__ddiv_rn(fp.kappa * (r - fp.r_coll), r) + __ddiv_rn(fp.eta * rv, r2));
    cn[0] += fc * dx;
    cn[1] += fc * dy;
    cn[2] += fc * dz;
}

// Contact term only (gravity already counted by the FP32 loop).
__device__ __forceinline__ void contact64(const ForceParams& fp, const double* __restrict__ x,
                                          const double* __restrict__ y, const double* __restrict__ z,
                                          const double* __restrict__ vx, const double* __restrict__ vy,
                                          const double* __restrict__ vz, const double* __restrict__ m,
                                          int64_t i, int64_t j, double* cn) {
    const double dx = __dsub_rn(x[j], x[i]), dy = __dsub_rn(y[j], y[i]), dz = __dsub_rn(z[j], z[i]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (r2 == 0.0 || r2 > fp.rc2) return;
    const double r = __dsqrt_rn(r2);
    const double dvx = __dsub_rn(vx[j], vx[i]), dvy = __dsub_rn(vy[j], vy[i]), dvz = __dsub_rn(vz[j], vz[i]);
    const double rv = __dadd_rn(__dadd_rn(__dmul_rn(dx, dvx), __dmul_rn(dy, dvy)), __dmul_rn(dz, dvz));
    const double mi = m[i], mj = m[j];
    const double fc = __ddiv_rn(mj, __dadd_rn(mi, mj)) *
                      (__ddiv_rn(fp.kappa * (r - fp.r_coll), r) + __ddiv_rn(fp.eta * rv, r2));
    cn[0] += fc * dx;
    cn[1] += fc * dy;
    cn[2] += fc * dz;
}

__device__ __forceinline__ void central64(double G_Mc, double x, double y, double z, double* a) {
    const double r2 = x * x + y * y + z * z;
    const double f = -G_Mc / (r2 * sqrt(r2));
    a[0] += f * x;
    a[1] += f * y;
    a[2] += f * z;
}

// ---------------------------------------------------------------------------
// FP64 kernel
// ---------------------------------------------------------------------------
constexpr int kWarps = 4;

struct __align__(32) D4 {
    double x, y, z, w;
};

struct Smem64 {
    D4 pj[32];
    uint32_t jid[32];
    double cl[32][10];  // M, c3, Q6
};

__global__ void __launch_bounds__(32 * kWarps) k_force64(
    int64_t ng, const int32_t* __restrict__ groups, const uint32_t* __restrict__ begin,
    const uint32_t* __restrict__ end, const int64_t* __restrict__ jj_off, const uint32_t* __restrict__ JJ,
    const int64_t* __restrict__ pc_off, const int32_t* __restrict__ C, const double* __restrict__ x,
    const double* __restrict__ y, const double* __restrict__ z, const double* __restrict__ vx,
    const double* __restrict__ vy, const double* __restrict__ vz, const double* __restrict__ m,
    const double* __restrict__ M, const double* __restrict__ cx, const double* __restrict__ cy,
    const double* __restrict__ cz, const double* __restrict__ Q, ForceParams fp, bool add_central,
    double* __restrict__ ax, double* __restrict__ ay, double* __restrict__ az, uint32_t n, int64_t nn,
    int* status) {
    __shared__ Smem64 sm[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * kWarps + w;
    if (k >= ng) return;
    Smem64& S = sm[w];
    const int32_t g = groups[k];
    const uint32_t b = begin[g], e = end[g];
    const int64_t j0 = jj_off[k], j1 = jj_off[k + 1], c0 = pc_off[k], c1 = pc_off[k + 1];
    for (uint32_t i0 = b; i0 < e; i0 += 32) {
        const uint32_t i = i0 + lane;
        const bool valid = i < e;
        const uint32_t ii = valid ? i : b;
        const double xi = x[ii], yi = y[ii], zi = z[ii];
        double ag[3] = {0.0, 0.0, 0.0}, an[3] = {0.0, 0.0, 0.0};
        for (int64_t t0 = j0; t0 < j1; t0 += 32) {
            const int nt = (int)min((int64_t)32, j1 - t0);
            if (lane < nt) {
                uint32_t j = JJ[t0 + lane];
                if (j >= n) {
                    atomicOr(status, kStatBounds);
                    j = b;
                }
                S.pj[lane] = D4{x[j], y[j], z[j], m[j]};
                S.jid[lane] = j;
            }
            __syncwarp();
            for (int q = 0; q < nt; ++q) {
                const D4 pj = S.pj[q];
                const double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > fp.rc2_hi) {
                    const double s2 = r2 + fp.eps2;
                    const double ri = rsqrt(s2);
                    const double f = pj.w * ri * ri * ri;
                    ag[0] += f * dx;
                    ag[1] += f * dy;
                    ag[2] += f * dz;
                } else {
                    const uint32_t j = S.jid[q];
                    if (valid && j != i)
                        near_pair64(fp, xi, yi, zi, vx[ii], vy[ii], vz[ii], m[ii], pj.x, pj.y, pj.z, vx[j],
                                    vy[j], vz[j], pj.w, ag, an);
                }
            }
            __syncwarp();
        }
        for (int64_t t0 = c0; t0 < c1; t0 += 32) {
            const int nt = (int)min((int64_t)32, c1 - t0);
            if (lane < nt) {
                int32_t cc = C[t0 + lane];
                if (cc < 0 || cc >= nn) {
                    atomicOr(status, kStatBounds);
                    cc = 0;
                }
                S.cl[lane][0] = M[cc];
                S.cl[lane][1] = cx[cc];
                S.cl[lane][2] = cy[cc];
                S.cl[lane][3] = cz[cc];
                if (fp.order >= 2)
#pragma unroll
                    for (int a = 0; a < 6; ++a) S.cl[lane][4 + a] = Q[6 * (int64_t)cc + a];
            }
            __syncwarp();
            for (int q = 0; q < nt; ++q) {
                const double* cl = S.cl[q];
                const double dx = cl[1] - xi, dy = cl[2] - yi, dz = cl[3] - zi;  // d = c - x_i = -R
                const double R2 = dx * dx + dy * dy + dz * dz + fp.eps2;
                const double ri = rsqrt(R2);
                const double ri2 = ri * ri;
                const double ri3 = ri * ri2;
                const double mono = cl[0] * ri3;
                ag[0] += mono * dx;
                ag[1] += mono * dy;
                ag[2] += mono * dz;
                if (fp.order >= 2) {
                    const double qx = cl[4] * dx + cl[7] * dy + cl[8] * dz;
                    const double qy = cl[7] * dx + cl[5] * dy + cl[9] * dz;
                    const double qz = cl[8] * dx + cl[9] * dy + cl[6] * dz;
                    const double dqd = dx * qx + dy * qy + dz * qz;
                    const double ri5 = ri3 * ri2;
                    const double s = 2.5 * dqd * ri2;
                    ag[0] += ri5 * (s * dx - qx);
                    ag[1] += ri5 * (s * dy - qy);
                    ag[2] += ri5 * (s * dz - qz);
                }
            }
            __syncwarp();
        }
        if (valid) {
            double a[3] = {fp.G * ag[0] + an[0], fp.G * ag[1] + an[1], fp.G * ag[2] + an[2]};
            if (add_central) central64(fp.GMc, xi, yi, zi, a);
            ax[i] = a[0];
            ay[i] = a[1];
            az[i] = a[2];
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 group-relative kernel
// ---------------------------------------------------------------------------
constexpr int kR = 2;  // i-particles per lane

struct Smem32 {
    float4 pj[32];
    uint32_t jid[32];
    float4 cl[32][3];  // (c_rel, M), (Qxx, Qxy, Qxz, Qyy), (Qyz, -, -, -)
};

__device__ __forceinline__ float rel(float hi, float lo, float ohi, float olo) {
    return __fadd_rn(__fsub_rn(hi, ohi), __fsub_rn(lo, olo));
}

template <int ORDER, bool MASK0>
__global__ void __launch_bounds__(32 * kWarps) k_force32(
    int64_t ng, const int32_t* __restrict__ groups, const uint32_t* __restrict__ begin,
    const uint32_t* __restrict__ end, const int64_t* __restrict__ jj_off, const uint32_t* __restrict__ JJ,
    const int64_t* __restrict__ pc_off, const int32_t* __restrict__ C, const float4* __restrict__ phi,
    const float4* __restrict__ plo, const float4* __restrict__ cell32, const double* __restrict__ cx,
    const double* __restrict__ cy, const double* __restrict__ cz, const double* __restrict__ x,
    const double* __restrict__ y, const double* __restrict__ z, const double* __restrict__ vx,
    const double* __restrict__ vy, const double* __restrict__ vz, const double* __restrict__ m,
    ForceParams fp, bool add_central, double* __restrict__ ax, double* __restrict__ ay,
    double* __restrict__ az, uint32_t n, int64_t nn, int* status) {
    __shared__ Smem32 sm[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * kWarps + w;
    if (k >= ng) return;
    Smem32& S = sm[w];
    const int32_t g = groups[k];
    const uint32_t b = begin[g], e = end[g];
    const int64_t j0 = jj_off[k], j1 = jj_off[k + 1], c0 = pc_off[k], c1 = pc_off[k + 1];
    // group origin: FP64 centre of mass of the group node, split hi/lo
    float oh[3], ol[3];
    {
        const double o[3] = {cx[g], cy[g], cz[g]};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            oh[a] = __double2float_rn(o[a]);
            ol[a] = __double2float_rn(__dsub_rn(o[a], (double)oh[a]));
        }
    }
    for (uint32_t i0 = b; i0 < e; i0 += 32 * kR) {
        float xr[kR], yr[kR], zr[kR], acx[kR], acy[kR], acz[kR];
        uint32_t iv[kR];
        bool vl[kR];
        double an[kR][3];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const uint32_t i = i0 + r * 32 + lane;
            vl[r] = i < e;
            iv[r] = vl[r] ? i : b;
            const float4 h = phi[iv[r]], l = plo[iv[r]];
            xr[r] = rel(h.x, l.x, oh[0], ol[0]);
            yr[r] = rel(h.y, l.y, oh[1], ol[1]);
            zr[r] = rel(h.z, l.z, oh[2], ol[2]);
            acx[r] = acy[r] = acz[r] = 0.f;
            an[r][0] = an[r][1] = an[r][2] = 0.0;
        }
        for (int64_t t0 = j0; t0 < j1; t0 += 32) {
            const int nt = (int)min((int64_t)32, j1 - t0);
            if (lane < nt) {
                uint32_t j = JJ[t0 + lane];
                if (j >= n) {
                    atomicOr(status, kStatBounds);
                    j = b;
                }
                const float4 h = phi[j], l = plo[j];
                S.pj[lane] = make_float4(rel(h.x, l.x, oh[0], ol[0]), rel(h.y, l.y, oh[1], ol[1]),
                                         rel(h.z, l.z, oh[2], ol[2]), h.w);
                S.jid[lane] = j;
            }
            __syncwarp();
            for (int q = 0; q < nt; ++q) {
                const float4 pj = S.pj[q];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const float dx = pj.x - xr[r], dy = pj.y - yr[r], dz = pj.z - zr[r];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float s2 = fmaxf(r2 + fp.eps2f, fp.floor2f);
                    const float ri = rsqrt_approx(s2);
                    float f = pj.w * ri * (ri * ri);
                    if (MASK0) f = r2 > 0.f ? f : 0.f;
                    acx[r] = fmaf(f, dx, acx[r]);
                    acy[r] = fmaf(f, dy, acy[r]);
                    acz[r] = fmaf(f, dz, acz[r]);
                    if (r2 <= fp.rc2chk_f) {
                        const uint32_t j = S.jid[q];
                        if (vl[r] && j != iv[r]) contact64(fp, x, y, z, vx, vy, vz, m, iv[r], j, an[r]);
                    }
                }
            }
            __syncwarp();
        }
        for (int64_t t0 = c0; t0 < c1; t0 += 32) {
            const int nt = (int)min((int64_t)32, c1 - t0);
            if (lane < nt) {
                int32_t cc = C[t0 + lane];
                if (cc < 0 || cc >= nn) {
                    atomicOr(status, kStatBounds);
                    cc = 0;
                }
                const float4 r0 = cell32[3 * (int64_t)cc], r1 = cell32[3 * (int64_t)cc + 1];
                S.cl[lane][0] = make_float4(rel(r0.x, r1.x, oh[0], ol[0]), rel(r0.y, r1.y, oh[1], ol[1]),
                                            rel(r0.z, r1.z, oh[2], ol[2]), r0.w);
                if (ORDER >= 2) {
                    const float4 r2v = cell32[3 * (int64_t)cc + 2];  // Qxy, Qxz, Qyy, Qyz
                    S.cl[lane][1] = make_float4(r1.w, r2v.x, r2v.y, r2v.z);
                    S.cl[lane][2] = make_float4(r2v.w, 0.f, 0.f, 0.f);
                }
            }
            __syncwarp();
            for (int q = 0; q < nt; ++q) {
                const float4 c4 = S.cl[q][0];
                float4 qa, qb;
                if (ORDER >= 2) {
                    qa = S.cl[q][1];
                    qb = S.cl[q][2];
                }
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const float dx = c4.x - xr[r], dy = c4.y - yr[r], dz = c4.z - zr[r];
                    const float R2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, fp.eps2f)));
                    const float ri = rsqrt_approx(R2);
                    const float ri2 = ri * ri;
                    const float ri3 = ri * ri2;
                    if (ORDER >= 2) {
                        // Q = [[xx, xy, xz], [xy, yy, yz], [xz, yz, -(xx+yy)]]
                        const float qzz = -(qa.x + qa.w);
                        const float qx = fmaf(qa.x, dx, fmaf(qa.y, dy, qa.z * dz));
                        const float qy = fmaf(qa.y, dx, fmaf(qa.w, dy, qb.x * dz));
                        const float qz = fmaf(qa.z, dx, fmaf(qb.x, dy, qzz * dz));
                        const float dqd = fmaf(dx, qx, fmaf(dy, qy, dz * qz));
                        const float ri5 = ri3 * ri2;
                        const float s = fmaf(2.5f * dqd, ri5 * ri2, c4.w * ri3);
                        acx[r] = fmaf(s, dx, fmaf(-ri5, qx, acx[r]));
                        acy[r] = fmaf(s, dy, fmaf(-ri5, qy, acy[r]));
                        acz[r] = fmaf(s, dz, fmaf(-ri5, qz, acz[r]));
                    } else {
                        const float s = c4.w * ri3;
                        acx[r] = fmaf(s, dx, acx[r]);
                        acy[r] = fmaf(s, dy, acy[r]);
                        acz[r] = fmaf(s, dz, acz[r]);
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            if (!vl[r]) continue;
            const uint32_t i = iv[r];
            double a[3] = {fp.G * (double)acx[r] + an[r][0], fp.G * (double)acy[r] + an[r][1],
                           fp.G * (double)acz[r] + an[r][2]};
            if (add_central) central64(fp.GMc, x[i], y[i], z[i], a);
            ax[i] = a[0];
            ay[i] = a[1];
            az[i] = a[2];
        }
    }
}

__global__ void k_split_particles(const double* __restrict__ x, const double* __restrict__ y,
                                  const double* __restrict__ z, const double* __restrict__ m, int64_t n,
                                  float4* __restrict__ phi, float4* __restrict__ plo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v[3] = {x[i], y[i], z[i]};
    float h[3], l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        h[a] = __double2float_rn(v[a]);
        l[a] = __double2float_rn(__dsub_rn(v[a], (double)h[a]));
    }
    phi[i] = make_float4(h[0], h[1], h[2], __double2float_rn(m[i]));
    plo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

ForceParams force_params(const Ctx* c) {
    const bh_params& p = c->prm;
    ForceParams fp;
    fp.G = p.G;
    fp.eps2 = p.eps * p.eps;
    fp.rc2 = p.r_coll * p.r_coll;
    fp.rc2_hi = fp.rc2 * (1.0 + 1e-10);
    fp.kappa = p.kappa;
    fp.eta = p.eta;
    fp.r_coll = p.r_coll;
    fp.GMc = p.G * p.M_central;
    fp.eps2f = (float)fp.eps2;
    fp.floor2f = (float)(fp.rc2 + fp.eps2);
    fp.rc2chk_f = (float)(fp.rc2 * 1.02);
    fp.order = p.order;
    return fp;
}

}  // namespace

int stage_split(Ctx* c, const bh_particles* p) {
    BH_TRY(grow(c, c->phi, (size_t)c->n, "FP32 positions hi"));
    BH_TRY(grow(c, c->plo, (size_t)c->n, "FP32 positions lo"));
    k_split_particles<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(p->x, p->y, p->z, p->m, c->n, c->phi.p,
                                                                    c->plo.p);
    BH_LAUNCH(c);
    return BH_OK;
}

int stage_force(Ctx* c, bh_particles* p, bool add_central) {
    const int64_t ng = c->n_groups;
    const ForceParams fp = force_params(c);
    const unsigned nb = blocks_for(ng, kWarps);
    add_central = add_central && c->prm.M_central != 0.0;
    if (c->prm.precision == BH_PREC_FP64) {
        k_force64<<<nb, 32 * kWarps, 0, c->stream>>>(ng, c->groups.p, c->begin.p, c->end.p, c->cnt_j.p, c->JJ.p,
                                                     c->cnt_c.p, c->C.p, p->x, p->y, p->z, p->vx, p->vy, p->vz,
                                                     p->m, c->M.p, c->cx.p, c->cy.p, c->cz.p, c->Q.p, fp,
                                                     add_central, p->ax, p->ay, p->az, (uint32_t)c->n,
                                                     c->n_nodes, c->d_status);
        BH_LAUNCH(c);
        return BH_OK;
    }
    BH_TRY(stage_split(c, p));
    const bool mask0 = !(fp.floor2f > 0.f);
#define BH_F32(O, MK)                                                                                         \
    k_force32<O, MK><<<nb, 32 * kWarps, 0, c->stream>>>(                                                     \
        ng, c->groups.p, c->begin.p, c->end.p, c->cnt_j.p, c->JJ.p, c->cnt_c.p, c->C.p, c->phi.p, c->plo.p,   \
        c->cell32.p, c->cx.p, c->cy.p, c->cz.p, p->x, p->y, p->z, p->vx, p->vy, p->vz, p->m, fp, add_central, \
        p->ax, p->ay, p->az, (uint32_t)c->n, c->n_nodes, c->d_status)
    if (c->prm.order >= 2) {
        if (mask0) BH_F32(2, true); else BH_F32(2, false);
    } else {
        if (mask0) BH_F32(1, true); else BH_F32(1, false);
    }
#undef BH_F32
    BH_LAUNCH(c);
    return BH_OK;
}

}  // namespace bh
