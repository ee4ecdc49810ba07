// force.cu -- Sec. 4.2 step 3d, second half: the double loop over the
// particles of a group and the entries of its shared interaction list.
//
//   list particles: Eq. (1) read as an acceleration (gravity G m_j r/r^3,
//                   softened by eps, held at its r_coll value inside r_coll,
//                   plus the spring/dashpot contact term inside r_coll);
//   list cells:     centre-of-mass monopole (Sec. 5.1) and, for order 2, the
//                   traceless quadrupole about the centre of mass.
//
// This file: the plain FP64 kernel (absolute coordinates, one warp per group,
// list entries staged 32 at a time in shared memory and broadcast to the
// lanes), the per-evaluation FP32 hi/lo split used by the FP32 kernel
// (force32.cu), and the dispatcher.  Pairs that may be in contact
// (r^2 <= r_coll^2 up to rounding) are re-evaluated in the oracle's exact
// operation order, so the r <= r_coll decision is the oracle's.
#include <cmath>

#include "force_common.cuh"
#include "split32.cuh"

namespace bh {
namespace {

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
    int64_t ng, const unsigned long long* __restrict__ dng, const unsigned long long* __restrict__ abort,
    const int32_t* __restrict__ groups, const uint32_t* __restrict__ begin,
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
    if (dng) ng = min(ng, (int64_t)*dng);  // device-sized list build
    if (k >= ng || (abort && *abort)) return;  // (abort: that build outgrew its buffers)
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
        // the group's own particles first (segment 0), then the other list particles
        for (int seg = 0; seg < 2; ++seg) {
            const int64_t s0 = seg == 0 ? (int64_t)b : j0, s1 = seg == 0 ? (int64_t)e : j1;
            for (int64_t t0 = s0; t0 < s1; t0 += 32) {
                const int nt = (int)min((int64_t)32, s1 - t0);
                if (lane < nt) {
                    uint32_t j = seg == 0 ? (uint32_t)(t0 + lane) : JJ[t0 + lane];
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
                            exact_pair64(fp, xi, yi, zi, vx[ii], vy[ii], vz[ii], m[ii], pj.x, pj.y, pj.z, vx[j],
                                         vy[j], vz[j], pj.w, an);
                    }
                }
                __syncwarp();
            }
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


// Self-gravity potential of every particle over its group's lists, FP64:
// the potential of the gravity Eq. (1) applies (held at its r_coll value
// inside r_coll) for the group's own particles (j != i) and the list
// particles, then the monopole + quadrupole potential of the list cells.
// Same staging as k_force64.
__global__ void __launch_bounds__(32 * kWarps) k_potential64(
    int64_t ng, const int32_t* __restrict__ groups, const uint32_t* __restrict__ begin,
    const uint32_t* __restrict__ end, const int64_t* __restrict__ jj_off, const uint32_t* __restrict__ JJ,
    const int64_t* __restrict__ pc_off, const int32_t* __restrict__ C, const double* __restrict__ x,
    const double* __restrict__ y, const double* __restrict__ z, const double* __restrict__ m,
    const double* __restrict__ M, const double* __restrict__ cx, const double* __restrict__ cy,
    const double* __restrict__ cz, const double* __restrict__ Q, ForceParams fp, double* __restrict__ phi,
    uint32_t n, int64_t nn, int* status) {
    __shared__ Smem64 sm[kWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * kWarps + w;
    if (k >= ng) return;
    Smem64& S = sm[w];
    const int32_t g = groups[k];
    const uint32_t b = begin[g], e = end[g];
    const int64_t j0 = jj_off[k], j1 = jj_off[k + 1], c0 = pc_off[k], c1 = pc_off[k + 1];
    const double s2c = fp.rc2 + fp.eps2, sc = sqrt(s2c);
    for (uint32_t i0 = b; i0 < e; i0 += 32) {
        const uint32_t i = i0 + lane;
        const bool valid = i < e;
        const uint32_t ii = valid ? i : b;
        const double xi = x[ii], yi = y[ii], zi = z[ii];
        double acc = 0.0;
        for (int seg = 0; seg < 2; ++seg) {
            const int64_t s0 = seg == 0 ? (int64_t)b : j0, s1 = seg == 0 ? (int64_t)e : j1;
            for (int64_t t0 = s0; t0 < s1; t0 += 32) {
                const int nt = (int)min((int64_t)32, s1 - t0);
                if (lane < nt) {
                    uint32_t j = seg == 0 ? (uint32_t)(t0 + lane) : JJ[t0 + lane];
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
                    if (S.jid[q] == i) continue;
                    const double dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0) continue;
                    if (r2 > fp.rc2)
                        acc -= pj.w / sqrt(r2 + fp.eps2);
                    else
                        acc -= pj.w / sc + pj.w * (fp.rc2 - r2) / (2.0 * s2c * sc);
                }
                __syncwarp();
            }
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
                const double Rx = xi - cl[1], Ry = yi - cl[2], Rz = zi - cl[3];
                const double R2 = Rx * Rx + Ry * Ry + Rz * Rz + fp.eps2;
                const double R = sqrt(R2);
                acc -= cl[0] / R;
                if (fp.order >= 2) {
                    const double qx = cl[4] * Rx + cl[7] * Ry + cl[8] * Rz;
                    const double qy = cl[7] * Rx + cl[5] * Ry + cl[9] * Rz;
                    const double qz = cl[8] * Rx + cl[9] * Ry + cl[6] * Rz;
                    acc -= 0.5 * (Rx * qx + Ry * qy + Rz * qz) / (R2 * R2 * R);
                }
            }
            __syncwarp();
        }
        if (valid) phi[i] = fp.G * acc;
    }
}

// W = 1/2 sum m_i phi_i in a fixed order (fixed grid, grid-stride loops,
// block tree, one final pass), so repeated calls give the same bits.
constexpr int kWBlocks = 512, kWThreads = 256;

__global__ void __launch_bounds__(kWThreads) k_wsum_partial(int64_t n, const double* __restrict__ m,
                                                            const double* __restrict__ phi, double* part) {
    __shared__ double sh[kWThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kWThreads + threadIdx.x; i < n; i += (int64_t)kWBlocks * kWThreads)
        acc += 0.5 * m[i] * phi[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kWThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_wsum_final(const double* __restrict__ part, double* out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < kWBlocks; ++b) s += part[b];
    *out = s;
}

__global__ void k_split_particles(const double* __restrict__ x, const double* __restrict__ y,
                                  const double* __restrict__ z, const double* __restrict__ m, int64_t n,
                                  float4* __restrict__ phi, float4* __restrict__ plo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v[3] = {x[i], y[i], z[i]};
    float h[3], l[3], mh, ml;
#pragma unroll
    for (int a = 0; a < 3; ++a) split_f32(v[a], h[a], l[a]);
    split_f32(m[i], mh, ml);
    phi[i] = make_float4(h[0], h[1], h[2], mh);
    plo[i] = make_float4(l[0], l[1], l[2], ml);
}

// The split alone, for callers and tests of it (bh_split_f32).
__global__ void k_split_values(const double* __restrict__ v, int64_t n, float* __restrict__ hi,
                               float* __restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h, l;
    split_f32(v[i], h, l);
    hi[i] = h;
    lo[i] = l;
}

}  // namespace

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
    fp.rc2f = (float)fp.rc2;
    fp.kappaf = (float)p.kappa;
    fp.etaf = (float)p.eta;
    fp.rcollf = (float)p.r_coll;
    fp.Gf = (float)p.G;
    fp.order = p.order;
    return fp;
}

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
    add_central = add_central && c->prm.M_central != 0.0;
    if (c->prm.precision == BH_PREC_FP64) {
        const unsigned nb = blocks_for(ng, kWarps);
        BH_TRY(timing_begin(c));
        BH_TRY(stage_begin(c, BH_STAGE_FORCE));
        const unsigned long long* dng = c->dev_build ? c->d_sz + kSzNg : nullptr;
        k_force64<<<nb, 32 * kWarps, 0, c->stream>>>(ng, dng, c->abort, c->groups.p, c->begin.p, c->end.p, c->cnt_j.p, c->JJ.p,
                                                     c->cnt_c.p, c->C.p, p->x, p->y, p->z, p->vx, p->vy, p->vz,
                                                     p->m, c->M.p, c->cx.p, c->cy.p, c->cz.p, c->Q.p, fp,
                                                     add_central, p->ax, p->ay, p->az, (uint32_t)c->n,
                                                     c->n_nodes, c->d_status);
        BH_LAUNCH(c);
        BH_TRY(stage_end(c));
        return timing_end(c);
    }
    // the hi/lo split and the FP32 records were made by stage_moments
    return launch_force32(c, p, fp, add_central);
}

int stage_potential(Ctx* c, const bh_particles* p, double* phi, double* W) {
    BH_TRY(stage_moments64(c, p));  // FP64 moments of the current positions, either precision
    if (!phi) {
        BH_TRY(grow(c, c->pot, (size_t)c->n, "potential"));
        phi = c->pot.p;
    }
    const ForceParams fp = force_params(c);
    k_potential64<<<blocks_for(c->n_groups, kWarps), 32 * kWarps, 0, c->stream>>>(
        c->n_groups, c->groups.p, c->begin.p, c->end.p, c->cnt_j.p, c->JJ.p, c->cnt_c.p, c->C.p, p->x, p->y, p->z,
        p->m, c->M.p, c->cx.p, c->cy.p, c->cz.p, c->Q.p, fp, phi, (uint32_t)c->n, c->n_nodes, c->d_status);
    BH_LAUNCH(c);
    if (W) {
        BH_TRY(grow(c, c->diag, (size_t)kWBlocks + 1, "potential energy sums"));
        k_wsum_partial<<<kWBlocks, kWThreads, 0, c->stream>>>(c->n, p->m, phi, c->diag.p);
        BH_LAUNCH(c);
        k_wsum_final<<<1, 32, 0, c->stream>>>(c->diag.p, c->diag.p + kWBlocks);
        BH_LAUNCH(c);
        BH_CUDA(c, cudaMemcpyAsync(W, c->diag.p + kWBlocks, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return BH_OK;
}

}  // namespace bh

extern "C" int bh_split_f32(const double* v, float* hi, float* lo, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!v || !hi || !lo)) || (n > 0 && hi == lo)) return BH_E_INVAL;
    if (n == 0) return BH_OK;
    bh::k_split_values<<<bh::blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(v, n, hi, lo);
    return cudaGetLastError() == cudaSuccess ? BH_OK : BH_E_CUDA;
}
