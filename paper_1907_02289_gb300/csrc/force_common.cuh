// force_common.cuh -- pieces shared by the FP64 and FP32 force kernels:
// parameters, the exact FP64 pair term of Eq. (1) and the central mass.
#pragma once
#include "bh_internal.cuh"

namespace bh {

struct ForceParams {
    double G, eps2, rc2, rc2_hi, kappa, eta, r_coll, GMc;
    float eps2f, rc2f, kappaf, etaf, rcollf, Gf;
    int order;
};

ForceParams force_params(const Ctx* c);
int launch_force32(Ctx* c, bh_particles* p, const ForceParams& fp, bool add_central);

// Eq. (1) for one pair, FP64, in the oracle's operation order (no
// contraction): returns the acceleration of i (gravity includes G).
// Coincident positions contribute nothing.
__device__ __forceinline__ void exact_pair64(const ForceParams& fp, double xi, double yi, double zi,
                                             double vxi, double vyi, double vzi, double mi, double xj,
                                             double yj, double zj, double vxj, double vyj, double vzj,
                                             double mj, double* a) {
    const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (r2 == 0.0) return;
    double f;
    if (r2 > fp.rc2) {
        const double s2 = __dadd_rn(r2, fp.eps2);
        f = __ddiv_rn(__dmul_rn(fp.G, mj), __dmul_rn(s2, __dsqrt_rn(s2)));
    } else {
        const double s2 = __dadd_rn(fp.rc2, fp.eps2);
        const double r = __dsqrt_rn(r2);
        const double dvx = __dsub_rn(vxj, vxi), dvy = __dsub_rn(vyj, vyi), dvz = __dsub_rn(vzj, vzi);
        const double rv = __dadd_rn(__dadd_rn(__dmul_rn(dx, dvx), __dmul_rn(dy, dvy)), __dmul_rn(dz, dvz));
        f = __dadd_rn(__ddiv_rn(__dmul_rn(fp.G, mj), __dmul_rn(s2, __dsqrt_rn(s2))),
                      __dmul_rn(__ddiv_rn(mj, __dadd_rn(mi, mj)),
                                __dadd_rn(__ddiv_rn(__dmul_rn(fp.kappa, __dsub_rn(r, fp.r_coll)), r),
                                          __ddiv_rn(__dmul_rn(fp.eta, rv), r2))));
    }
    a[0] += f * dx;
    a[1] += f * dy;
    a[2] += f * dz;
}

// The spring and dashpot part of Eq. (1) alone (the gravity at r_coll is
// added elsewhere): nonzero iff 0 < r <= r_coll, decided in FP64 in the
// oracle's operation order.
__device__ __forceinline__ bool contact_term64(const ForceParams& fp, double xi, double yi, double zi, double vxi,
                                               double vyi, double vzi, double mi, double xj, double yj, double zj,
                                               double vxj, double vyj, double vzj, double mj, double* a) {
    const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (r2 == 0.0 || r2 > fp.rc2) return false;
    const double r = __dsqrt_rn(r2);
    const double dvx = __dsub_rn(vxj, vxi), dvy = __dsub_rn(vyj, vyi), dvz = __dsub_rn(vzj, vzi);
    const double rv = __dadd_rn(__dadd_rn(__dmul_rn(dx, dvx), __dmul_rn(dy, dvy)), __dmul_rn(dz, dvz));
    const double f = __dmul_rn(__ddiv_rn(mj, __dadd_rn(mi, mj)),
                               __dadd_rn(__ddiv_rn(__dmul_rn(fp.kappa, __dsub_rn(r, fp.r_coll)), r),
                                         __ddiv_rn(__dmul_rn(fp.eta, rv), r2)));
    a[0] += f * dx;
    a[1] += f * dy;
    a[2] += f * dz;
    return true;
}

// Central mass at the origin: a += -G Mc x / |x|^3.
__device__ __forceinline__ void central64(double G_Mc, double x, double y, double z, double* a) {
    const double r2 = x * x + y * y + z * z;
    const double f = -G_Mc / (r2 * sqrt(r2));
    a[0] += f * x;
    a[1] += f * y;
    a[2] += f * z;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

}  // namespace bh
