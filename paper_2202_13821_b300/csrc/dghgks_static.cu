// dghgks_residual_static: one residual evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc/cudaFree at the point where they need a
// residual: code that runs inside another framework's memory plan (a caching
// allocator that already owns the free device memory, or a fixed budget
// planned at start-up), real-time or embedded loops that forbid allocation
// after initialisation, and code that must not trigger the implicit device
// synchronisation that cudaFree performs.  dghgks_init allocates its scratch
// (stage buffers and face moments) with cudaMalloc, so such callers cannot
// use a context.  This entry point needs no context: its only scratch, the
// face moments of the residual, lives in a file-scope __device__ array of
// fixed size, which every GPU that loads the library holds until the process
// exits.
//
// Host code must not pass the array's name to a kernel (in host code the
// name is a host-side stand-in, not a device address): the first call on
// each device looks up the device address with cudaGetSymbolAddress, with
// that device current, and every launch uses that address.
#include <cuda_runtime.h>

#include <mutex>

#include "dg_kernels.cuh"
#include "dghgks.h"

using namespace dghgks;

namespace {

constexpr size_t kScratchBytes = (size_t)DGHGKS_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) unsigned g_flag;

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;
  unsigned* flag = nullptr;
};
DeviceSetup g_dev[kMaxDevices];
std::mutex g_dev_mu;

template <class R, int ORDER, int NQ>
cudaError_t set_attrs() {
  using FS = FaceSmem<R, ORDER, NQ>;
  cudaError_t e = cudaSuccess;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_face<R, ORDER, NQ, 0, double>, a, (int)FS::bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_face<R, ORDER, NQ, 1, double>, a, (int)FS::bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_face<R, ORDER, NQ, 2, double>, a, (int)FS::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cell<R, ORDER, NQ, MODE_RESIDUAL, double>, a, (int)CellSmem<R, ORDER, NQ, double>::bytes);
  return e;
}

// Once per device, with that device current: device addresses of the static
// scratch and flag, and the shared-memory attributes of the kernels.
int setup_current_device(DeviceSetup** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DGHGKS_ECUDA;
  std::lock_guard<std::mutex> lock(g_dev_mu);
  DeviceSetup& d = g_dev[dev];
  if (!d.done) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DGHGKS_ECUDA;
    d.scratch = static_cast<unsigned char*>(p);
    p = nullptr;
    if (cudaGetSymbolAddress(&p, g_flag) != cudaSuccess || !p) return DGHGKS_ECUDA;
    d.flag = static_cast<unsigned*>(p);
    cudaError_t e = set_attrs<double, 1, 2>();
    if (e == cudaSuccess) e = set_attrs<double, 2, 2>();
    if (e == cudaSuccess) e = set_attrs<double, 2, 3>();
    if (e == cudaSuccess) e = set_attrs<float, 1, 2>();
    if (e == cudaSuccess) e = set_attrs<float, 2, 2>();
    if (e == cudaSuccess) e = set_attrs<float, 2, 3>();
    if (e != cudaSuccess) return DGHGKS_ECUDA;
    d.done = true;
  }
  *out = &d;
  return DGHGKS_OK;
}

template <class R, int ORDER, int NQ>
void launch(const MeshDev& m, const GasPar<R>& g, const double* Q, double* L, double* Lt, R* G, unsigned* flag,
            double dt, cudaStream_t s) {
  using FS = FaceSmem<R, ORDER, NQ>;
  using LY = CellLayout<ORDER, NQ>;
  const dim3 fgrid((m.nx + FB - 1) / FB, m.ny, m.nz), fblock(FS::THREADS);
  k_face<R, ORDER, NQ, 0, double><<<fgrid, fblock, FS::bytes, s>>>(Q, G, g, m, flag);
  k_face<R, ORDER, NQ, 1, double><<<fgrid, fblock, FS::bytes, s>>>(Q, G, g, m, flag);
  k_face<R, ORDER, NQ, 2, double><<<fgrid, fblock, FS::bytes, s>>>(Q, G, g, m, flag);
  StageIO<R> io;
  io.L = L;
  io.Lt = Lt;
  io.Qs = nullptr;
  io.inc = nullptr;
  io.Qn = nullptr;
  io.Qf = nullptr;
  dim3 cgrid;
  size_t csmem = 0;
  cell_launch_config<R, ORDER, NQ, MODE_RESIDUAL, double>(m, cgrid, csmem);
  k_cell<R, ORDER, NQ, MODE_RESIDUAL, double><<<cgrid, LY::WARPS * 32, csmem, s>>>(Q, G, io, g, m, dt, flag);
}

template <class R>
GasPar<R> gas(double gamma, double mu, double Pr, double tau_eps, double dt) {
  GasPar<R> g;
  g.K = (R)((5.0 - 3.0 * gamma) / (gamma - 1.0));
  g.gm1 = (R)(gamma - 1.0);
  g.mu = (R)mu;
  g.tau_add = (R)(tau_eps * dt);
  g.pr_fix = (R)(1.0 / Pr - 1.0);
  g.dt = (R)dt;
  g.inv_dt = (R)(1.0 / dt);
  return g;
}

}  // namespace

extern "C" int dghgks_residual_static(const dghgks_mesh* mesh, int order, double gamma, double mu, double Pr,
                                      const dghgks_opts* opts, const double* Q, double dt, double* L, double* Lt,
                                      void* stream) {
  if (!mesh || !Q || !L || !Lt) return DGHGKS_EARG;
  if (L == Q || Lt == Q || L == Lt) return DGHGKS_EARG;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || mesh->ny > 65535 || mesh->nz > 65535) return DGHGKS_EARG;
  for (int d = 0; d < 3; ++d) {
    if (!(mesh->hi[d] > mesh->lo[d])) return DGHGKS_EARG;
    if (mesh->periodic[d] != 1) return DGHGKS_EUNSUP;
    if (mesh->nodes[d]) return DGHGKS_EUNSUP;  // uniform meshes only
  }
  if (!(gamma > 1.0) || !(mu >= 0.0) || !(Pr > 0.0) || !(dt > 0.0)) return DGHGKS_EARG;
  const int nq = (opts && opts->n_q) ? opts->n_q : order + 1;
  const int precision = opts ? opts->precision : DGHGKS_FP64;
  const double tau_eps = opts ? opts->tau_eps : 0.0;
  if (precision != DGHGKS_FP64 && precision != DGHGKS_FP32_MIXED) return DGHGKS_EARG;
  if (!(tau_eps >= 0.0)) return DGHGKS_EARG;
  if (!((order == 1 && nq == 2) || (order == 2 && (nq == 2 || nq == 3)))) return DGHGKS_EUNSUP;

  // the face moments must fit the static scratch
  const long long ncell = (long long)mesh->nx * mesh->ny * mesh->nz;
  const size_t rsize = precision == DGHGKS_FP64 ? sizeof(double) : sizeof(float);
  const size_t need = rsize * 30 * (size_t)n_tmodes(order) * (size_t)ncell;
  if (need > kScratchBytes) return DGHGKS_ESCRATCH;

  DeviceSetup* d = nullptr;
  if (int rc = setup_current_device(&d)) return rc;

  MeshDev m;
  m.nx = mesh->nx;
  m.ny = mesh->ny;
  m.nz = mesh->nz;
  m.ncell = ncell;
  m.vol = 1.0;
  const int n3[3] = {mesh->nx, mesh->ny, mesh->nz};
  for (int k = 0; k < 3; ++k) {
    m.h[k] = (mesh->hi[k] - mesh->lo[k]) / n3[k];
    m.vol *= m.h[k];
  }
  for (int k = 0; k < 3; ++k) {
    m.sc_f[k] = (float)(2.0 / m.h[k]);
    m.area_f[k] = (float)(m.vol / m.h[k]);
  }
  m.vol_f = (float)m.vol;
  m.ivol = 1.0 / m.vol;
  m.ivol_f = (float)(1.0 / m.vol);
  for (int k = 0; k < 3; ++k) {
    m.geo64[k] = nullptr;
    m.geo32[k] = nullptr;
  }

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the flag must start at zero: it keeps the previous call's value
  if (cudaMemsetAsync(d->flag, 0, sizeof(unsigned), s) != cudaSuccess) return DGHGKS_ECUDA;
  if (precision == DGHGKS_FP64) {
    const GasPar<double> g = gas<double>(gamma, mu, Pr, tau_eps, dt);
    double* G = reinterpret_cast<double*>(d->scratch);
    if (order == 1) launch<double, 1, 2>(m, g, Q, L, Lt, G, d->flag, dt, s);
    else if (nq == 2) launch<double, 2, 2>(m, g, Q, L, Lt, G, d->flag, dt, s);
    else launch<double, 2, 3>(m, g, Q, L, Lt, G, d->flag, dt, s);
  } else {
    const GasPar<float> g = gas<float>(gamma, mu, Pr, tau_eps, dt);
    float* G = reinterpret_cast<float*>(d->scratch);
    if (order == 1) launch<float, 1, 2>(m, g, Q, L, Lt, G, d->flag, dt, s);
    else if (nq == 2) launch<float, 2, 2>(m, g, Q, L, Lt, G, d->flag, dt, s);
    else launch<float, 2, 3>(m, g, Q, L, Lt, G, d->flag, dt, s);
  }
  if (cudaGetLastError() != cudaSuccess) return DGHGKS_ECUDA;
  unsigned flag = 0;
  if (cudaMemcpyAsync(&flag, d->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return DGHGKS_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DGHGKS_ECUDA;
  if (flag & 2u) return DGHGKS_ECUDA;  // a kernel-internal barrier wait timed out
  return flag ? DGHGKS_EPHYS : DGHGKS_OK;
}
