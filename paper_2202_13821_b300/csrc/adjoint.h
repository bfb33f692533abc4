// Internal interface between the C-ABI layer (dghgks_api.cu) and the adjoint
// kernels (dghgks_adjoint.cu, compiled as a separate translation unit).
#pragma once
#include <cuda_runtime.h>

#include "dg_kernels.cuh"

namespace dghgks {

// Adjoint scratch of one stage: face cotangents H[D][side][comp][face]
// (side 0 = left cell of the face, 1 = right cell; comp = v * NM + n).
struct AdjIO {
  const double* lamA;  // first cotangent input (state layout)
  const double* lamB;  // second cotangent input (may be NULL)
  double cLA, cLB;     // lambda_L  = cLA lamA + cLB lamB
  double cTA, cTB;     // lambda_Lt = cTA lamA + cTB lamB
  double* H;           // face cotangents
  double* out;         // cotangent of Q (state layout)
  const double* addA;  // out = addA + addB + J^T lambda (either may be NULL)
  const double* addB;
  double* mu_part;     // per-CTA partial sums of the viscosity cotangent
};

// shared-memory attributes of the adjoint kernels of (order, n_q)
cudaError_t adjoint_set_attrs(int order, int nq);
// one residual VJP (3 face launches + 1 cell launch); mu partials at io.mu_part
// CTAs of one face-VJP launch (their viscosity partials are indexed by CTA)
long long adjoint_face_ctas(int order, int nx, int ny, int nz);
void adjoint_vjp(int order, int nq, const double* Q, const GasPar<double>& g, const MeshDev& m, const AdjIO& io,
                 cudaStream_t s);
// *acc += sum of the n partials (fixed order)
void adjoint_mu_sum(const double* part, long long n, double* acc, cudaStream_t s);
// gradient of E_k with respect to Q (scale = |K| / (rho0 |Omega|))
// dE_k/dQ; scale = 1/(rho0 |Omega|) times |K| on a uniform mesh (a rectilinear mesh weights each cell by its volume)
void adjoint_ek_vjp(int order, int nq, const double* Q, const MeshDev& m, double scale, double* out, cudaStream_t s);
// number of launches one adjoint_vjp makes
constexpr int kAdjointLaunches = 4;

}  // namespace dghgks
