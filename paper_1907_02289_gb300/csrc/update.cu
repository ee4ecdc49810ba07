// update.cu -- Sec. 4.2 step 4 ("integrate the orbits"): the FP64
// kick-drift-kick leapfrog.  The acceleration arrays already hold the tree
// part plus the central mass (added by the force kernel's epilogue).
#include "bh_internal.cuh"

namespace bh {
namespace {

__global__ void k_kick(int64_t n, double h, const double* __restrict__ ax, const double* __restrict__ ay,
                       const double* __restrict__ az, double* __restrict__ vx, double* __restrict__ vy,
                       double* __restrict__ vz) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vx[i] += h * ax[i];
    vy[i] += h * ay[i];
    vz[i] += h * az[i];
}

__global__ void k_kick_drift(int64_t n, double h, double dt, const double* __restrict__ ax,
                             const double* __restrict__ ay, const double* __restrict__ az,
                             double* __restrict__ vx, double* __restrict__ vy, double* __restrict__ vz,
                             double* __restrict__ x, double* __restrict__ y, double* __restrict__ z) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ux = vx[i] + h * ax[i], uy = vy[i] + h * ay[i], uz = vz[i] + h * az[i];
    vx[i] = ux;
    vy[i] = uy;
    vz[i] = uz;
    x[i] += dt * ux;
    y[i] += dt * uy;
    z[i] += dt * uz;
}

}  // namespace

int stage_kick(Ctx* c, bh_particles* p, double h) {
    k_kick<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(c->n, h, p->ax, p->ay, p->az, p->vx, p->vy, p->vz);
    BH_LAUNCH(c);
    return BH_OK;
}

int stage_kick_drift(Ctx* c, bh_particles* p, double h, double dt) {
    k_kick_drift<<<blocks_for(c->n, 256), 256, 0, c->stream>>>(c->n, h, dt, p->ax, p->ay, p->az, p->vx, p->vy,
                                                               p->vz, p->x, p->y, p->z);
    BH_LAUNCH(c);
    return BH_OK;
}

}  // namespace bh
