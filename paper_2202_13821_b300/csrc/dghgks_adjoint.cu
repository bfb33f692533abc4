// Adjoint (VJP) kernels of the DG-HGKS residual and their launchers.  This
// translation unit is compiled with -Xptxas -O1: at -O3 ptxas caps the face
// VJP (one long reverse sweep per Gauss point) at 96 registers with 17 KB of
// spills per thread; at -O1 it uses 168 registers and spills 7.6 KB.  The
// forward kernels stay in dghgks_api.cu at -O3.
#include "adjoint.h"
#include "dg_adjoint.cuh"

namespace dghgks {

namespace {
constexpr int kRedBlocksAdj = 148 * 8;

template <int ORDER, int NQ, bool FTO>
cudaError_t attrs_k() {
  cudaError_t e = cudaSuccess;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int fb = (int)FaceAdjSmem<ORDER, NQ>::bytes, cb = (int)CellAdjSmem<ORDER, NQ>::bytes;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_face_vjp<ORDER, NQ, 0, FTO>, a, fb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_face_vjp<ORDER, NQ, 1, FTO>, a, fb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_face_vjp<ORDER, NQ, 2, FTO>, a, fb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cell_vjp<ORDER, NQ, FTO>, a, cb);
  return e;
}
template <int ORDER, int NQ>
cudaError_t attrs() {
  const cudaError_t e = attrs_k<ORDER, NQ, false>();
  return e == cudaSuccess ? attrs_k<ORDER, NQ, true>() : e;
}

template <int ORDER, int NQ, bool FTO>
void vjp_k(const double* Q, const GasPar<double>& g, const MeshDev& m, const AdjIO& io, cudaStream_t s) {
  constexpr int FBA = adj_fb<ORDER>();
  const dim3 fgrid((m.nx + FBA - 1) / FBA, m.ny, m.nz), fblock(FBA * NQ * NQ);
  const size_t fblocks = (size_t)fgrid.x * fgrid.y * fgrid.z;
  const size_t fbytes = FaceAdjSmem<ORDER, NQ>::bytes;
  k_face_vjp<ORDER, NQ, 0, FTO><<<fgrid, fblock, fbytes, s>>>(Q, g, m, io, 0 * fblocks);
  k_face_vjp<ORDER, NQ, 1, FTO><<<fgrid, fblock, fbytes, s>>>(Q, g, m, io, 1 * fblocks);
  k_face_vjp<ORDER, NQ, 2, FTO><<<fgrid, fblock, fbytes, s>>>(Q, g, m, io, 2 * fblocks);
  using LY = CellLayout<ORDER, NQ>;
  const dim3 cgrid((m.nx + LY::CB - 1) / LY::CB, m.ny, m.nz), cblock(LY::WARPS * 32);
  k_cell_vjp<ORDER, NQ, FTO><<<cgrid, cblock, CellAdjSmem<ORDER, NQ>::bytes, s>>>(Q, g, m, io, 3 * fblocks);
}
// a zero cotangent of L (stage 2 of the S2O4 adjoint) takes the F_t-only sweeps
template <int ORDER, int NQ>
void vjp(const double* Q, const GasPar<double>& g, const MeshDev& m, const AdjIO& io, cudaStream_t s) {
  if (io.cLA == 0.0 && io.cLB == 0.0)
    vjp_k<ORDER, NQ, true>(Q, g, m, io, s);
  else
    vjp_k<ORDER, NQ, false>(Q, g, m, io, s);
}
}  // namespace

cudaError_t adjoint_set_attrs(int order, int nq) {
  if (order == 1 && nq == 2) return attrs<1, 2>();
  if (order == 2 && nq == 2) return attrs<2, 2>();
  if (order == 2 && nq == 3) return attrs<2, 3>();
  if (order == 3 && nq == 3) return attrs<3, 3>();
  if (order == 3 && nq == 4) return attrs<3, 4>();
  return cudaErrorInvalidValue;
}

void adjoint_vjp(int order, int nq, const double* Q, const GasPar<double>& g, const MeshDev& m, const AdjIO& io,
                 cudaStream_t s) {
  if (order == 1 && nq == 2) vjp<1, 2>(Q, g, m, io, s);
  else if (order == 2 && nq == 2) vjp<2, 2>(Q, g, m, io, s);
  else if (order == 2 && nq == 3) vjp<2, 3>(Q, g, m, io, s);
  else if (order == 3 && nq == 3) vjp<3, 3>(Q, g, m, io, s);
  else if (order == 3 && nq == 4) vjp<3, 4>(Q, g, m, io, s);
}

long long adjoint_face_ctas(int order, int nx, int ny, int nz) {
  const int fb = order >= 3 ? adj_fb<3>() : adj_fb<1>();
  return (long long)((nx + fb - 1) / fb) * ny * nz;
}

void adjoint_mu_sum(const double* part, long long n, double* acc, cudaStream_t s) {
  k_mu_sum<<<1, RED_THREADS, 0, s>>>(part, n, acc);
}

void adjoint_ek_vjp(int order, int nq, const double* Q, const MeshDev& m, double scale, double* out,
                    cudaStream_t s) {
  if (order == 1 && nq == 2) k_ek_vjp<1, 2><<<kRedBlocksAdj, RED_THREADS, 0, s>>>(Q, m, scale, out);
  else if (order == 2 && nq == 2) k_ek_vjp<2, 2><<<kRedBlocksAdj, RED_THREADS, 0, s>>>(Q, m, scale, out);
  else if (order == 2 && nq == 3) k_ek_vjp<2, 3><<<kRedBlocksAdj, RED_THREADS, 0, s>>>(Q, m, scale, out);
  else if (order == 3 && nq == 3) k_ek_vjp<3, 3><<<kRedBlocksAdj, RED_THREADS, 0, s>>>(Q, m, scale, out);
  else if (order == 3 && nq == 4) k_ek_vjp<3, 4><<<kRedBlocksAdj, RED_THREADS, 0, s>>>(Q, m, scale, out);
}

}  // namespace dghgks
