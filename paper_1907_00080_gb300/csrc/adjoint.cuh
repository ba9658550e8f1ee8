// Arguments of the reverse-mode (adjoint) step kernels (adjoint_kernels.cu).
//
// One FP64 time step maps S^n = (d*^{n-1}, X^n, X^{n-1}) to S^{n+1}; its
// adjoint maps the adjoints of S^{n+1} to those of S^n and adds the step's
// share of dJ/dk_s, dJ/dk_b and dJ/dsigma.  The primal quantities of step n
// (forces, shape functions and their stencils, the spread force field) are the
// ones the context's own step computed, copied to the tape when the segment
// is re-run; areas and bounding boxes are re-evaluated from X^n.  The bond set
// of step n is the recorded one (bond events are not differentiated).
#pragma once

#include "tangent.cuh"

namespace lbib {

struct AdjointArgs {
    TangentArgs t;        // primal state of step n: t.f = d*^{n-1}, t.m.X = X^n, t.m.bond_of_lig = bonds
                          // of step n, t.Fv = F^n, t.Wv = shape functions, t.st = stencil origins (wrapped
                          // i0, j0), all from the tape; t.A, t.Ad, t.box filled by the area kernel
    const longlong2* gfix;  // [N] spread force of step n, fixed point (scaled by 2^52)
    const double* fbar;   // [9][N] adjoint of d*^n (the deviations step n stores)
    double* fbar_out;     // [9][N] adjoint of d*^{n-1}; every entry is written
    const double* XB;     // [nv][2] adjoint of X^{n+1}
    double* XB_out;       // [nv][2] adjoint of X^n (written by k_a_interp, then accumulated)
    double* XPB;          // [nv][2] in: adjoint of X^n as the previous position of step n+1;
                          //          out: adjoint of X^{n-1}
    double* ubar;         // [N][2] adjoint of the interpolated velocity field (zero between steps)
    double* Gbar;         // [N][2] adjoint of the spread force
    double* Wbar;         // [nv][9] adjoint of the shape functions
    double* Abar;         // [nmem] adjoint of the enclosed areas
    double* ks_bar;       // [nmem] accumulated dJ/dk_s
    double* kb_bar;       // [nmem] accumulated dJ/dk_b
    double* sigma_bar;    // [1] accumulated dJ/dsigma
};

cudaError_t launch_adjoint_step(const AdjointArgs& a, cudaStream_t s);

// enclosed areas A[k][nmem] and bounding boxes box[k][nmem][4] of the taped
// positions X_k = tape_X + k * 2 nv of steps k = 0 .. len-1, in one launch
cudaError_t launch_tape_areas(const MarkerArgs& m, const double* tape_X, int len, double* A, double* box,
                              cudaStream_t s);

// Up to four device-to-device copies of whole 4-byte words in one launch (the
// tape of a step: fewer calls per reverse step than one copy each)
struct CopyList {
    const void* src[4];
    void* dst[4];
    size_t words[4];
    int n;
};
cudaError_t launch_copy_words(const CopyList& l, cudaStream_t s);

// FP64 copies for the tape of a context of another precision: stored
// populations (deviations, scaled storage undone) and compute-type arrays
cudaError_t launch_widen_storage(lbib_precision prec, const void* src, double* dst, size_t n, float inv_scale,
                                 cudaStream_t s);
cudaError_t launch_widen_compute(lbib_precision prec, const void* src, double* dst, size_t n, cudaStream_t s);

// adjoint of the stored deviations <-> adjoint of the pre-collision
// populations in the read-back layout (f^n_i(x) = w_i + d*_i(source of (x, i)))
cudaError_t launch_adjoint_perm(const double* in, double* out, int nx, int ny, int walls, int to_storage,
                                cudaStream_t s);

}  // namespace lbib
