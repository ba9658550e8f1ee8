// Arguments of the tangent-linear step kernels (tangent_kernels.cu).
#pragma once

#include "lbib_internal.cuh"

namespace lbib {

struct TangentArgs {
    MarkerArgs m;          // the primal context's marker state (FP64): X^n, X^{n-1}, bonds of step n
    const double* f;       // primal post-collision deviations of step n-1 [9][N]
    const double* fd_src;  // their tangent [9][N]
    double* fd_dst;        // tangent of the deviations this step stores [9][N]
    const double* dX;      // tangent of X^n [nv][2]
    const double* dXp;     // tangent of X^{n-1}
    double* dXn;           // tangent of X^{n+1}
    double *Gv, *Gd;       // [N][2] spread IB force and its tangent (zeroed per step)
    double *u, *ud;        // [N][2] u^n and its tangent
    double *Wv, *Wd;       // [nv][9] shape functions and tangents
    int* st;               // [nv][2] stencil origin (i0, j0), unwrapped
    double *Fv, *Fd;       // [nv][2] marker forces and tangents
    double *A, *Ad;        // [nmem] enclosed areas and tangents
    double* box;           // [nmem][4] bounding box of X^n: x_min, x_max, y_min, y_max
    const double* dks;     // [nmem] tangent of k_s per membrane
    const double* dkb;     // [nmem] tangent of k_b per membrane
    double dsigma;         // tangent of the bond stiffness
    const double* th0;     // [nv] rest turning angle at each vertex (Eq. bendFor's theta_0)
    const double* l0;      // [nv] rest length of element (v, v+1) (Eq. strainFor's l_0)
    double omega, gx, gy;
    long long step;        // n (forward Euler at n = 0)
};

cudaError_t launch_tangent_step(const TangentArgs& t, cudaStream_t s);
// the marker part alone (areas and boxes, forces, shape functions, spreading
// into t.Gv / t.Gd, which the caller has zeroed)
cudaError_t launch_tangent_markers(const TangentArgs& t, cudaStream_t s);
// enclosed areas (value and tangent) and bounding boxes of X^n alone
cudaError_t launch_tangent_areas(const TangentArgs& t, cudaStream_t s);
// rest lengths l0[nv] and turning angles th0[nv] = atan2(cross, dot) of the
// context's rest records, in FP64 whatever the context's precision
cudaError_t launch_rest_fp64(lbib_precision prec, const MarkerArgs& m, double* l0, double* th0, cudaStream_t s);

}  // namespace lbib
