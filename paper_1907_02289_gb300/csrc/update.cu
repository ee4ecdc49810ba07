// update.cu -- Sec. 4.2 step 4 ("integrate the orbits"): the FP64
// kick-drift-kick leapfrog.  The acceleration arrays already hold the tree
// part plus the central mass (added by the force kernel's epilogue).
#include <cmath>

#include "bh_internal.cuh"

namespace bh {
namespace {

// abort (a list-constructing graph step): nonzero overflow bits mean the
// step's forces were not computed, so the kick is skipped.
__global__ void k_kick(int64_t n, double h, const double* __restrict__ ax, const double* __restrict__ ay,
                       const double* __restrict__ az, double* __restrict__ vx, double* __restrict__ vy,
                       double* __restrict__ vz, const unsigned long long* __restrict__ abort) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || (abort && *abort)) return;
    vx[i] += h * ax[i];
    vy[i] += h * ay[i];
    vz[i] += h * az[i];
}

// Kick and drift; with ROT the frame then turns by omega dt (Sec. 4.4): x, y
// and vx, vy are rotated by -omega dt about z (c = cos, s = sin of omega dt),
// each product rounded on its own, as the oracle's step does.
template <bool ROT>
__global__ void k_kick_drift(int64_t n, double h, double dt, const double* __restrict__ ax,
                             const double* __restrict__ ay, const double* __restrict__ az,
                             double* __restrict__ vx, double* __restrict__ vy, double* __restrict__ vz,
                             double* __restrict__ x, double* __restrict__ y, double* __restrict__ z, double c,
                             double s) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ux = vx[i] + h * ax[i], uy = vy[i] + h * ay[i], uz = vz[i] + h * az[i];
    const double X = x[i] + dt * ux, Y = y[i] + dt * uy;
    z[i] += dt * uz;
    vz[i] = uz;
    if (ROT) {
        x[i] = __dadd_rn(__dmul_rn(c, X), __dmul_rn(s, Y));
        y[i] = __dsub_rn(__dmul_rn(c, Y), __dmul_rn(s, X));
        vx[i] = __dadd_rn(__dmul_rn(c, ux), __dmul_rn(s, uy));
        vy[i] = __dsub_rn(__dmul_rn(c, uy), __dmul_rn(s, ux));
    } else {
        x[i] = X;
        y[i] = Y;
        vx[i] = ux;
        vy[i] = uy;
    }
}

// Diagnostics: 11 FP64 sums per particle set (mass, momentum, angular
// momentum about the origin, kinetic energy, central-mass potential energy),
// reduced in a fixed order (fixed grid, grid-stride loops, fixed block
// tree, one final block), so the result is bit-reproducible.
constexpr int kDiagSums = 11, kDiagBlocks = 512, kDiagThreads = 256;

__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(
    int64_t n, double GMc, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
    const double* __restrict__ vx, const double* __restrict__ vy, const double* __restrict__ vz,
    const double* __restrict__ m, double* __restrict__ part) {
    __shared__ double sh[kDiagSums][kDiagThreads];
    double acc[kDiagSums];
#pragma unroll
    for (int q = 0; q < kDiagSums; ++q) acc[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kDiagThreads + threadIdx.x; i < n; i += (int64_t)kDiagBlocks * kDiagThreads) {
        const double mi = m[i], X = x[i], Y = y[i], Z = z[i], U = vx[i], V = vy[i], W = vz[i];
        acc[0] += mi;
        acc[1] += mi * U;
        acc[2] += mi * V;
        acc[3] += mi * W;
        acc[4] += mi * (Y * W - Z * V);
        acc[5] += mi * (Z * U - X * W);
        acc[6] += mi * (X * V - Y * U);
        acc[7] += 0.5 * mi * (U * U + V * V + W * W);
        const double r = sqrt(X * X + Y * Y + Z * Z);
        acc[8] += r > 0.0 ? -GMc * mi / r : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kDiagSums; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < kDiagSums; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kDiagSums) part[(int64_t)blockIdx.x * kDiagSums + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void k_diag_final(const double* __restrict__ part, double* out) {
    const int q = threadIdx.x;
    if (q >= kDiagSums) return;
    double s = 0.0;
    for (int b = 0; b < kDiagBlocks; ++b) s += part[(int64_t)b * kDiagSums + q];
    out[q] = s;
}

}  // namespace

int stage_diagnostics(Ctx* c, const bh_particles* p, double* host_out) {
    BH_TRY(grow(c, c->diag, (size_t)kDiagBlocks * kDiagSums + kDiagSums, "diagnostic sums"));
    double* part = c->diag.p;
    double* out = part + (size_t)kDiagBlocks * kDiagSums;
    k_diag_partial<<<kDiagBlocks, kDiagThreads, 0, c->stream>>>(p->n, c->prm.G * c->prm.M_central, p->x, p->y, p->z,
                                                                 p->vx, p->vy, p->vz, p->m, part);
    BH_LAUNCH(c);
    k_diag_final<<<1, 32, 0, c->stream>>>(part, out);
    BH_LAUNCH(c);
    BH_CUDA(c, cudaMemcpyAsync(host_out, out, kDiagSums * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    return BH_OK;
}

int stage_kick(Ctx* c, bh_particles* p, double h) {
    BH_TRY(stage_begin(c, BH_STAGE_UPDATE));
    k_kick<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(c->n, h, p->ax, p->ay, p->az, p->vx, p->vy, p->vz,
                                                         c->abort);
    BH_LAUNCH(c);
    return stage_end(c);
}

int stage_kick_drift(Ctx* c, bh_particles* p, double h, double dt) {
    BH_TRY(stage_begin(c, BH_STAGE_UPDATE));
    const double om = c->prm.omega * dt;
    auto kern = om != 0.0 ? k_kick_drift<true> : k_kick_drift<false>;
    kern<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(c->n, h, dt, p->ax, p->ay, p->az, p->vx, p->vy, p->vz, p->x,
                                                       p->y, p->z, std::cos(om), std::sin(om));
    BH_LAUNCH(c);
    return stage_end(c);
}

}  // namespace bh
