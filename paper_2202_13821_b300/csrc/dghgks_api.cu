// Host side of the C ABI declared in include/dghgks.h: context creation,
// scratch allocation, kernel dispatch over (precision, order, n_q), the S2O4
// driver and the FP64 reductions.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "adjoint.h"
#include "dg_kernels.cuh"
#include "dghgks.h"

using namespace dghgks;

namespace {

constexpr int kRedBlocks = 148 * 8;  // reduction grid: 8 CTAs per SM
constexpr int kProfMax = 65536;

struct Ops;

}  // namespace

struct dghgks_ctx {
  int device = 0;
  int n[3] = {0, 0, 0};
  long long ncell = 0;
  double lo[3], hi[3], h[3], vol = 0;
  double omega = 0;              // |Omega|
  bool nonuniform = false;       // rectilinear mesh given by node coordinates
  double* geo64 = nullptr;       // per axis: n_d widths, n_d values 2/width (device)
  float* geo32 = nullptr;        // the same in FP32
  int order = 0, nq = 0, nm = 0, nt = 0, precision = 0;
  double gamma = 1.4, K = 2.0, mu = 0, Pr = 1, tau_eps = 0;
  void* Qs = nullptr;   // Q* (stage-1 output), flux precision
  void* Qf = nullptr;   // FP32-mixed: the state rounded to FP32 by a stage-2 pass, read by the
                        // next step's stage-1 kernels within one dghgks_steps / dghgks_run_host call
  void* Inc = nullptr;  // dt L + dt^2/6 L_t (stage-1 output), epilogue precision (FP64 with
                        // DGHGKS_FP32_STAGE64, else the flux precision)
  void* G = nullptr;      // face moments [3][cells][10][NT] (face-major), flux precision
  unsigned* flag = nullptr;
  double* part = nullptr;  // reduction partials [kRedBlocks][5]
  double* red = nullptr;   // reduction results (device)
  double* red_host = nullptr;  // pinned
  double* Qdev = nullptr;      // device state for dghgks_run_host
  cudaStream_t ek_stream = nullptr;  // dghgks_run_host: E_k of step n beside step n+1
  cudaEvent_t ev_q = nullptr, ev_ek = nullptr;
  // adjoint scratch (FP64 contexts, allocated on first use)
  double* adjH = nullptr;      // face cotangents [3][2][5 N_m][cells]
  double* adjLam = nullptr;    // lambda* (state size)
  double* adjMu = nullptr;     // viscosity partials
  size_t adjMuN = 0;
  const Ops* ops = nullptr;
  int64_t launches = 0;
  // profiling: event pairs around launches
  bool prof = false;
  int prof_n = 0;
  cudaEvent_t* prof_ev = nullptr;  // [2 * kProfMax]
  int* prof_kind = nullptr;        // [kProfMax]
  // captured step graphs: [0] a step on the FP64 state, [1] a step on the FP32 copy
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  double* g_Q[2] = {nullptr, nullptr};  // arguments each captured graph was built with
  double g_dt[2] = {0.0, 0.0};
  double g_mu[2] = {-1.0, -1.0};
  bool g_out[2] = {false, false};
  char err[512] = {0};
};

namespace {

char g_init_err[512] = "";

int fail(dghgks_ctx* c, int code, const char* fmt, ...) {
  char* buf = c ? c->err : g_init_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_check(dghgks_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DGHGKS_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? DGHGKS_ENOMEM : DGHGKS_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

template <class R>
GasPar<R> gas_par(const dghgks_ctx* c, double dt) {
  GasPar<R> g;
  g.K = (R)c->K;
  g.gm1 = (R)(c->gamma - 1.0);
  g.mu = (R)c->mu;
  g.tau_add = (R)(c->tau_eps * dt);
  g.pr_fix = (R)(1.0 / c->Pr - 1.0);
  g.dt = (R)dt;
  g.inv_dt = (R)(1.0 / dt);
  return g;
}

MeshDev mesh_dev(const dghgks_ctx* c) {
  MeshDev m;
  m.nx = c->n[0];
  m.ny = c->n[1];
  m.nz = c->n[2];
  m.ncell = c->ncell;
  for (int d = 0; d < 3; ++d) {
    m.h[d] = c->h[d];
    m.sc_f[d] = (float)(2.0 / c->h[d]);
    m.area_f[d] = (float)(c->vol / c->h[d]);
  }
  m.vol = c->vol;
  m.vol_f = (float)c->vol;
  m.ivol = 1.0 / c->vol;
  m.ivol_f = (float)(1.0 / c->vol);
  int off = 0;
  for (int d = 0; d < 3; ++d) {
    m.geo64[d] = c->nonuniform ? c->geo64 + off : nullptr;
    m.geo32[d] = c->nonuniform ? c->geo32 + off : nullptr;
    off += 2 * c->n[d];
  }
  return m;
}

// Bracket one launch with profiling events when profiling is on.
struct ProfScope {
  dghgks_ctx* c;
  int slot = -1;
  cudaStream_t s;
  ProfScope(dghgks_ctx* c_, int kind, cudaStream_t s_) : c(c_), s(s_) {
    if (c->prof && c->prof_n < kProfMax) {
      slot = c->prof_n++;
      c->prof_kind[slot] = kind;
      cudaEventRecord(c->prof_ev[2 * slot], s);
    }
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(c->prof_ev[2 * slot + 1], s);
  }
};

enum { FACES_FP64 = 0, FACES_COPY = 1, FACES_QSTAR = 2 };

struct Ops {
  cudaError_t (*set_attrs)();
  // face pass: FACES_FP64 on the FP64 state, FACES_COPY on its FP32 copy Qf,
  // FACES_QSTAR the stage-2 pass on Q* (F_t moments only)
  void (*faces)(dghgks_ctx*, const void*, int, double, cudaStream_t);
  // cell pass: MODE_RESIDUAL (Q, L, Lt), MODE_STAGE1 (Q^n, or its copy Qf when
  // copy_in), MODE_STAGE2 (Q^n updated in place; Qf written when copy_out)
  void (*cell)(dghgks_ctx*, int, double*, double*, double*, double, cudaStream_t, bool copy_in, bool copy_out);
  void (*ek)(dghgks_ctx*, const double*, cudaStream_t);
  void (*enstrophy)(dghgks_ctx*, const double*, cudaStream_t);
  size_t r_size;  // flux precision: Q*, the FP32 state copy, face moments
  size_t e_size;  // epilogue precision: the stage increment inc
};

// E: precision of the cell kernels' epilogue (E = R, or double with R = float
// for the FP32-flux / FP64-stage contexts)
template <class R, int ORDER, int NQ, class E = R>
struct Impl {
  using FS = FaceSmem<R, ORDER, NQ>;

  static cudaError_t set_attrs() {
    cudaError_t e = cudaSuccess;
#define DG_ATTR(fn, bytes)                                                                         \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes));
    DG_ATTR((k_face<R, ORDER, NQ, 0, double>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 1, double>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 2, double>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 0, R, false>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 1, R, false>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 2, R, false>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 0, R, true>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 1, R, true>), FS::bytes)
    DG_ATTR((k_face<R, ORDER, NQ, 2, R, true>), FS::bytes)
    DG_ATTR((k_cell<R, ORDER, NQ, MODE_RESIDUAL, double, E>), (CellSmem<R, ORDER, NQ, double, E, MODE_RESIDUAL>::bytes))
    DG_ATTR((k_cell<R, ORDER, NQ, MODE_STAGE1, double, E>), (CellSmem<R, ORDER, NQ, double, E, MODE_STAGE1>::bytes))
    DG_ATTR((k_cell<R, ORDER, NQ, MODE_STAGE1, R, E>), (CellSmem<R, ORDER, NQ, R, E, MODE_STAGE1>::bytes))
    DG_ATTR((k_cell<R, ORDER, NQ, MODE_STAGE2, R, E>), (CellSmem<R, ORDER, NQ, R, E, MODE_STAGE2>::bytes))
#undef DG_ATTR
    return e;
  }

  template <class Tin, bool FTO>
  static void faces_t(dghgks_ctx* c, const Tin* Q, double dt, cudaStream_t s) {
    const GasPar<R> g = gas_par<R>(c, dt);
    const MeshDev m = mesh_dev(c);
    dim3 grid((c->n[0] + FB - 1) / FB, c->n[1], c->n[2]);
    dim3 block(FS::THREADS);
    R* G = static_cast<R*>(c->G);
    {
      ProfScope ps(c, 0, s);
      k_face<R, ORDER, NQ, 0, Tin, FTO><<<grid, block, FS::bytes, s>>>(Q, G, g, m, c->flag);
    }
    {
      ProfScope ps(c, 1, s);
      k_face<R, ORDER, NQ, 1, Tin, FTO><<<grid, block, FS::bytes, s>>>(Q, G, g, m, c->flag);
    }
    {
      ProfScope ps(c, 2, s);
      k_face<R, ORDER, NQ, 2, Tin, FTO><<<grid, block, FS::bytes, s>>>(Q, G, g, m, c->flag);
    }
    c->launches += 3;
  }

  static void faces(dghgks_ctx* c, const void* Q, int kind, double dt, cudaStream_t s) {
    if (kind == FACES_QSTAR)  // the stage-2 pass on Q*: F_t moments only
      faces_t<R, true>(c, static_cast<const R*>(Q), dt, s);
    else if (kind == FACES_COPY)
      faces_t<R, false>(c, static_cast<const R*>(Q), dt, s);
    else
      faces_t<double, false>(c, static_cast<const double*>(Q), dt, s);
  }

  template <int MODE, class Tin>
  static void cell_t(dghgks_ctx* c, const Tin* Qin, const R* G, const StageIO<R, E>& io, const GasPar<R>& g,
                     const MeshDev& m, double dt, cudaStream_t s) {
    dim3 grid;
    size_t smem = 0;
    cell_launch_config<R, ORDER, NQ, MODE, Tin, E>(m, grid, smem);
    k_cell<R, ORDER, NQ, MODE, Tin, E>
        <<<grid, CellLayout<ORDER, NQ>::WARPS * 32, smem, s>>>(Qin, G, io, g, m, dt, c->flag);
  }

  static void cell(dghgks_ctx* c, int mode, double* Q, double* L, double* Lt, double dt, cudaStream_t s,
                   bool copy_in, bool copy_out) {
    const GasPar<R> g = gas_par<R>(c, dt);
    const MeshDev m = mesh_dev(c);
    const R* G = static_cast<const R*>(c->G);
    StageIO<R, E> io;
    io.L = L;
    io.Lt = Lt;
    io.Qs = static_cast<R*>(c->Qs);
    io.inc = static_cast<E*>(c->Inc);
    io.Qn = Q;
    io.Qf = copy_out ? static_cast<R*>(c->Qf) : nullptr;
    ProfScope ps(c, 3 + mode, s);
    if (mode == MODE_RESIDUAL)
      cell_t<MODE_RESIDUAL, double>(c, Q, G, io, g, m, dt, s);
    else if (mode == MODE_STAGE1 && copy_in)
      cell_t<MODE_STAGE1, R>(c, static_cast<const R*>(c->Qf), G, io, g, m, dt, s);
    else if (mode == MODE_STAGE1)
      cell_t<MODE_STAGE1, double>(c, Q, G, io, g, m, dt, s);
    else
      cell_t<MODE_STAGE2, R>(c, io.Qs, G, io, g, m, dt, s);
    c->launches += 1;
  }

  static void enstrophy(dghgks_ctx* c, const double* Q, cudaStream_t s) {
    ProfScope ps(c, 6, s);
    k_enstrophy_part<ORDER, NQ><<<kRedBlocks, RED_THREADS, 0, s>>>(Q, mesh_dev(c), c->part);
    c->launches += 1;
  }

  static void ek(dghgks_ctx* c, const double* Q, cudaStream_t s) {
    ProfScope ps(c, 6, s);
    k_ek_part<ORDER, NQ><<<kRedBlocks, RED_THREADS, 0, s>>>(Q, mesh_dev(c), c->part);
    c->launches += 1;
  }
};

template <class R, int O, int N, class E = R>
constexpr Ops make_ops() {
  return Ops{&Impl<R, O, N, E>::set_attrs,
             &Impl<R, O, N, E>::faces,
             &Impl<R, O, N, E>::cell,
             &Impl<R, O, N, E>::ek,
             &Impl<R, O, N, E>::enstrophy,
             sizeof(R),
             sizeof(E)};
}
#define DG_OPS(R, O, N) make_ops<R, O, N>()
#define DG_OPS_STAGE64(O, N) make_ops<float, O, N, double>()

const Ops kOps64_1_2 = DG_OPS(double, 1, 2);
const Ops kOps64_2_2 = DG_OPS(double, 2, 2);
const Ops kOps64_2_3 = DG_OPS(double, 2, 3);
const Ops kOps32_1_2 = DG_OPS(float, 1, 2);
const Ops kOps32_2_2 = DG_OPS(float, 2, 2);
const Ops kOps32_2_3 = DG_OPS(float, 2, 3);
const Ops kOps64_3_3 = DG_OPS(double, 3, 3);
const Ops kOps64_3_4 = DG_OPS(double, 3, 4);
const Ops kOps32_3_3 = DG_OPS(float, 3, 3);
const Ops kOps32_3_4 = DG_OPS(float, 3, 4);
const Ops kOps32s_1_2 = DG_OPS_STAGE64(1, 2);
const Ops kOps32s_2_2 = DG_OPS_STAGE64(2, 2);
const Ops kOps32s_2_3 = DG_OPS_STAGE64(2, 3);
const Ops kOps32s_3_3 = DG_OPS_STAGE64(3, 3);
const Ops kOps32s_3_4 = DG_OPS_STAGE64(3, 4);

const Ops* select_ops(int precision, int order, int nq) {
  const int p = precision == DGHGKS_FP64 ? 0 : (precision == DGHGKS_FP32_MIXED ? 1 : 2);
  const Ops* const tab[5][3] = {{&kOps64_1_2, &kOps32_1_2, &kOps32s_1_2},
                                {&kOps64_2_2, &kOps32_2_2, &kOps32s_2_2},
                                {&kOps64_2_3, &kOps32_2_3, &kOps32s_2_3},
                                {&kOps64_3_3, &kOps32_3_3, &kOps32s_3_3},
                                {&kOps64_3_4, &kOps32_3_4, &kOps32s_3_4}};
  if (order == 1 && nq == 2) return tab[0][p];
  if (order == 2 && nq == 2) return tab[1][p];
  if (order == 2 && nq == 3) return tab[2][p];
  if (order == 3 && nq == 3) return tab[3][p];
  if (order == 3 && nq == 4) return tab[4][p];
  return nullptr;
}

// The state rounded to FP32 (round to nearest), the input of the stage-1
// kernels of FP32-mixed steps; n values, two per thread and step when both
// buffers are 16-byte aligned (VEC), else one.
template <bool VEC>
__global__ void __launch_bounds__(256) k_round_f32(const double* __restrict__ Q, float* __restrict__ Qf, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x, e0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (VEC) {
    for (size_t e = e0; e < n / 2; e += stride) {
      const double2 q = reinterpret_cast<const double2*>(Q)[e];
      reinterpret_cast<float2*>(Qf)[e] = make_float2((float)q.x, (float)q.y);
    }
    if (e0 == 0 && (n & 1)) Qf[n - 1] = (float)Q[n - 1];
  } else {
    for (size_t e = e0; e < n; e += stride) Qf[e] = (float)Q[e];
  }
}

template <int NM>
__global__ void __launch_bounds__(RED_THREADS) k_l2diff_part(const double* __restrict__ A, const double* __restrict__ B,
                                                             int var, const MeshDev m, double* __restrict__ part) {
  const long long nc = m.ncell;
  double acc[1] = {0};
  for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < nc; c += (long long)gridDim.x * RED_THREADS) {
    const double wc = cell_weight(m, c);
#pragma unroll
    for (int mm = 0; mm < NM; ++mm) {
      const size_t idx = (size_t)(var * NM + mm) * nc + c;
      const double d = A[idx] - B[idx];
      acc[0] += wc * (d * d / (double)((2 * mode_exp(mm, 0) + 1) * (2 * mode_exp(mm, 1) + 1) * (2 * mode_exp(mm, 2) + 1)));
    }
  }
  block_reduce_store<1>(acc, part);
}

// Final scale of the cell-sum reductions: the common cell volume on a uniform
// mesh; 1 on a rectilinear one, whose partial sums carry each cell's volume.
double vol_scale(const dghgks_ctx* c) { return c->nonuniform ? 1.0 : c->vol; }

int after_launch(dghgks_ctx* c, const char* what) { return cuda_check(c, cudaGetLastError(), what); }

int read_flag(dghgks_ctx* c, cudaStream_t s) {
  unsigned f = 0;
  int rc = cuda_check(c, cudaMemcpyAsync(&f, c->flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "flag read");
  if (rc) return rc;
  rc = cuda_check(c, cudaStreamSynchronize(s), "stream sync");
  if (rc) return rc;
  if (f) {
    cudaMemsetAsync(c->flag, 0, sizeof(unsigned), s);
    cudaStreamSynchronize(s);
    if (f & 2u) return fail(c, DGHGKS_ECUDA, "a barrier wait inside the cell kernel timed out (results invalid)");
    return fail(c, DGHGKS_EPHYS, "non-physical state (rho <= 0 or p <= 0) met at a quadrature point");
  }
  return DGHGKS_OK;
}

}  // namespace

extern "C" {

static void enqueue_step(dghgks_ctx* c, double* Q, double dt, cudaStream_t s, cudaEvent_t before_write,
                         bool have_copy = false, bool copy_out = false);

int dghgks_gauss_rule(int n, double* x, double* w) {
  if (n < 1 || n > 5 || !x || !w) return DGHGKS_EARG;
  for (int a = 0; a < n; ++a) {
    x[a] = gauss_x(n, a);
    w[a] = gauss_w(n, a);
  }
  return DGHGKS_OK;
}

int dghgks_init(const dghgks_mesh* mesh, int order, double gamma, double mu, double Pr, const dghgks_opts* opts,
                dghgks_ctx** out) {
  if (!out) return fail(nullptr, DGHGKS_EARG, "out is NULL");
  *out = nullptr;
  if (!mesh) return fail(nullptr, DGHGKS_EARG, "mesh is NULL");
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || mesh->ny > 65535 || mesh->nz > 65535)
    return fail(nullptr, DGHGKS_EARG, "bad mesh size %d x %d x %d", mesh->nx, mesh->ny, mesh->nz);
  const int n3[3] = {mesh->nx, mesh->ny, mesh->nz};
  // the cell kernels number their tiles of 8 cells in 32 bits
  if ((long long)((mesh->nx + 7) / 8) * mesh->ny * mesh->nz >= (1LL << 31))
    return fail(nullptr, DGHGKS_EUNSUP, "mesh of %d x %d x %d cells: too many cell tiles", mesh->nx, mesh->ny, mesh->nz);
  bool nonuniform = false;
  for (int d = 0; d < 3; ++d) {
    if (mesh->nodes[d]) {
      nonuniform = true;
      const double* x = mesh->nodes[d];
      for (int q = 0; q < n3[d]; ++q)
        if (!(std::isfinite(x[q]) && std::isfinite(x[q + 1]) && x[q + 1] > x[q]))
          return fail(nullptr, DGHGKS_EARG, "mesh nodes along axis %d not strictly increasing at %d", d, q);
    } else if (!(mesh->hi[d] > mesh->lo[d])) {
      return fail(nullptr, DGHGKS_EARG, "mesh hi <= lo along axis %d", d);
    }
    if (mesh->periodic[d] != 1) return fail(nullptr, DGHGKS_EUNSUP, "only periodic boundaries are supported");
  }
  if (!(gamma > 1.0) || !(mu >= 0.0) || !(Pr > 0.0)) return fail(nullptr, DGHGKS_EARG, "bad gas parameters");
  const int nq = (opts && opts->n_q) ? opts->n_q : order + 1;
  const int precision = opts ? opts->precision : DGHGKS_FP64;
  const double tau_eps = opts ? opts->tau_eps : 0.0;
  if (precision != DGHGKS_FP64 && precision != DGHGKS_FP32_MIXED && precision != DGHGKS_FP32_STAGE64)
    return fail(nullptr, DGHGKS_EARG, "precision must be DGHGKS_FP64, DGHGKS_FP32_MIXED or DGHGKS_FP32_STAGE64");
  if (!(tau_eps >= 0.0)) return fail(nullptr, DGHGKS_EARG, "tau_eps must be >= 0");
  const Ops* ops = select_ops(precision, order, nq);
  if (!ops) return fail(nullptr, DGHGKS_EUNSUP, "unsupported order %d with n_q %d", order, nq);

  dghgks_ctx* c = new (std::nothrow) dghgks_ctx();
  if (!c) return fail(nullptr, DGHGKS_ENOMEM, "host allocation failed");
  cudaGetDevice(&c->device);
  c->n[0] = mesh->nx;
  c->n[1] = mesh->ny;
  c->n[2] = mesh->nz;
  c->ncell = (long long)mesh->nx * mesh->ny * mesh->nz;
  c->vol = 1.0;
  c->nonuniform = nonuniform;
  // per-axis widths and 2/width of a rectilinear mesh (uniform axes filled
  // with their common width)
  std::vector<double> geo64;
  std::vector<float> geo32;
  for (int d = 0; d < 3; ++d) {
    const double* x = mesh->nodes[d];
    c->lo[d] = x ? x[0] : mesh->lo[d];
    c->hi[d] = x ? x[n3[d]] : mesh->hi[d];
    c->h[d] = (c->hi[d] - c->lo[d]) / c->n[d];
    c->vol *= c->h[d];
    if (nonuniform) {
      const size_t off = geo64.size();
      geo64.resize(off + 2 * n3[d]);
      for (int q = 0; q < n3[d]; ++q) {
        const double w = x ? x[q + 1] - x[q] : c->h[d];
        geo64[off + q] = w;
        geo64[off + n3[d] + q] = 2.0 / w;
      }
    }
  }
  c->omega = nonuniform ? (c->hi[0] - c->lo[0]) * (c->hi[1] - c->lo[1]) * (c->hi[2] - c->lo[2])
                        : c->vol * (double)c->ncell;
  for (double v : geo64) geo32.push_back((float)v);
  c->order = order;
  c->nq = nq;
  c->nm = n_modes(order);
  c->nt = n_tmodes(order);
  c->precision = precision;
  c->gamma = gamma;
  c->K = (5.0 - 3.0 * gamma) / (gamma - 1.0);
  c->mu = mu;
  c->Pr = Pr;
  c->tau_eps = tau_eps;
  c->ops = ops;

  const size_t stage = ops->r_size * 5 * (size_t)c->nm * c->ncell;
  const size_t stage_inc = ops->e_size * 5 * (size_t)c->nm * c->ncell;
  const size_t gbytes = ops->r_size * 30 * (size_t)c->nt * c->ncell;
  int rc = DGHGKS_OK;
  if (!rc) rc = cuda_check(c, ops->set_attrs(), "cudaFuncSetAttribute");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->Qs, stage), "cudaMalloc(Q*)");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->Inc, stage_inc), "cudaMalloc(stage increment)");
  if (!rc && precision != DGHGKS_FP64) rc = cuda_check(c, cudaMalloc(&c->Qf, stage), "cudaMalloc(FP32 state copy)");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->G, gbytes), "cudaMalloc(face moments)");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->flag, sizeof(unsigned)), "cudaMalloc(flag)");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->part, sizeof(double) * 5 * kRedBlocks), "cudaMalloc(partials)");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->red, sizeof(double) * 8), "cudaMalloc(red)");
  if (!rc) rc = cuda_check(c, cudaMallocHost(&c->red_host, sizeof(double) * 8), "cudaMallocHost");
  if (!rc) rc = cuda_check(c, cudaMemset(c->flag, 0, sizeof(unsigned)), "cudaMemset(flag)");
  if (!rc && nonuniform) {
    rc = cuda_check(c, cudaMalloc(&c->geo64, sizeof(double) * geo64.size()), "cudaMalloc(mesh widths)");
    if (!rc) rc = cuda_check(c, cudaMalloc(&c->geo32, sizeof(float) * geo32.size()), "cudaMalloc(mesh widths)");
    if (!rc)
      rc = cuda_check(c, cudaMemcpy(c->geo64, geo64.data(), sizeof(double) * geo64.size(), cudaMemcpyHostToDevice),
                      "copy mesh widths");
    if (!rc)
      rc = cuda_check(c, cudaMemcpy(c->geo32, geo32.data(), sizeof(float) * geo32.size(), cudaMemcpyHostToDevice),
                      "copy mesh widths");
  }
  if (rc) {
    snprintf(g_init_err, sizeof(g_init_err), "%s", c->err);
    dghgks_destroy(c);
    return rc;
  }
  *out = c;
  return DGHGKS_OK;
}

void dghgks_destroy(dghgks_ctx* c) {
  if (!c) return;
  for (int k = 0; k < 2; ++k)
    if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->prof_ev) {
    for (int e = 0; e < 2 * kProfMax; ++e) cudaEventDestroy(c->prof_ev[e]);
    delete[] c->prof_ev;
    delete[] c->prof_kind;
  }
  cudaFree(c->Qs);
  cudaFree(c->Qf);
  cudaFree(c->Inc);
  cudaFree(c->G);
  cudaFree(c->flag);
  cudaFree(c->part);
  cudaFree(c->red);
  cudaFree(c->Qdev);
  cudaFree(c->adjH);
  cudaFree(c->adjLam);
  cudaFree(c->adjMu);
  cudaFree(c->geo64);
  cudaFree(c->geo32);
  if (c->ev_q) cudaEventDestroy(c->ev_q);
  if (c->ev_ek) cudaEventDestroy(c->ev_ek);
  if (c->ek_stream) cudaStreamDestroy(c->ek_stream);
  if (c->red_host) cudaFreeHost(c->red_host);
  delete c;
}

const char* dghgks_last_error(const dghgks_ctx* c) { return c ? c->err : g_init_err; }

int dghgks_n_modes(const dghgks_ctx* c) { return c ? c->nm : DGHGKS_EARG; }

int64_t dghgks_launch_count(const dghgks_ctx* c) { return c ? c->launches : 0; }

int dghgks_set_mu(dghgks_ctx* c, double mu) {
  if (!c) return DGHGKS_EARG;
  if (!(mu >= 0.0)) return fail(c, DGHGKS_EARG, "mu must be >= 0");
  c->mu = mu;
  return DGHGKS_OK;
}

int dghgks_residual(dghgks_ctx* c, const double* Q, double dt, double* L, double* Lt, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q || !L || !Lt) return fail(c, DGHGKS_EARG, "NULL state or output pointer");
  if (!(dt > 0)) return fail(c, DGHGKS_EARG, "dt must be > 0");
  if (L == Q || Lt == Q || L == Lt) return fail(c, DGHGKS_EARG, "L, Lt and Q must be distinct buffers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->ops->faces(c, Q, FACES_FP64, dt, s);
  c->ops->cell(c, MODE_RESIDUAL, const_cast<double*>(Q), L, Lt, dt, s, false, false);
  return after_launch(c, "residual launch");
}

int dghgks_step(dghgks_ctx* c, double* Q, double dt, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q) return fail(c, DGHGKS_EARG, "Q is NULL");
  if (!(dt > 0)) return fail(c, DGHGKS_EARG, "dt must be > 0");
  // stage 1 at Q^n, stage 2 at Q* (same dt for the flux fit; only L_t(Q*) enters)
  enqueue_step(c, Q, dt, static_cast<cudaStream_t>(stream), nullptr);
  return after_launch(c, "step launch");
}

// Enqueue the 8 launches of one S2O4 step on s.  before_write (may be null): an event that the stage-2
// cell kernel, the only writer of Q, waits for (readers of Q^n on another
// stream).  FP32-mixed contexts: the stage-1 kernels always read the FP32
// copy Qf of Q^n (one set of kernels for every step, so results never depend
// on how the steps were grouped into calls); have_copy = the previous step of
// the same call wrote it, else Q^n is rounded into it first; copy_out = the
// stage-2 cell kernel writes Qf for the next step.
static void enqueue_step(dghgks_ctx* c, double* Q, double dt, cudaStream_t s, cudaEvent_t before_write,
                         bool have_copy, bool copy_out) {
  const bool copy = c->Qf != nullptr;
  if (copy && !have_copy) {
    const size_t n = 5 * (size_t)c->nm * c->ncell;
    const size_t blocks = (n / 2 + 255) / 256 < 4096 ? (n / 2 + 255) / 256 : 4096;
    const unsigned grid = (unsigned)(blocks ? blocks : 1);
    if (((uintptr_t)Q | (uintptr_t)c->Qf) % 16 == 0)
      k_round_f32<true><<<grid, 256, 0, s>>>(Q, static_cast<float*>(c->Qf), n);
    else  // the caller's state need only be 8-byte aligned
      k_round_f32<false><<<grid, 256, 0, s>>>(Q, static_cast<float*>(c->Qf), n);
    c->launches += 1;
  }
  c->ops->faces(c, copy ? c->Qf : Q, copy ? FACES_COPY : FACES_FP64, dt, s);
  c->ops->cell(c, MODE_STAGE1, Q, nullptr, nullptr, dt, s, copy, false);  // Q*, inc
  c->ops->faces(c, c->Qs, FACES_QSTAR, dt, s);
  if (before_write) cudaStreamWaitEvent(s, before_write, 0);
  c->ops->cell(c, MODE_STAGE2, Q, nullptr, nullptr, dt, s, false, copy && copy_out);  // Q += inc + dt^2/3 L_t(Q*)
}

// Capture (or update) step graph k: one step on Q, the first of a call (k = 0;
// on FP32-mixed contexts it rounds Q into the FP32 copy first) or a later one
// (k = 1, reading the copy the step before wrote), writing the copy when copy_out.
// The kernels' arguments (state pointer, dt and the gas parameters derived from
// dt and mu) are baked into the graph: capture again when one changed.
static int ensure_graph(dghgks_ctx* c, int k, double* Q, double dt, bool copy_out) {
  if (c->gexec[k] && c->g_Q[k] == Q && c->g_dt[k] == dt && c->g_mu[k] == c->mu && c->g_out[k] == copy_out)
    return DGHGKS_OK;
  const bool prof = c->prof;
  const int64_t launches = c->launches;
  c->prof = false;
  cudaGraph_t graph = nullptr;
  if (int rc = cuda_check(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "capture"))
    return rc;
  enqueue_step(c, Q, dt, c->cap_stream, nullptr, k == 1, copy_out);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  c->prof = prof;
  c->launches = launches;
  if (int rc = cuda_check(c, e, "end capture")) return rc;
  bool updated = false;
  if (c->gexec[k]) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(c->gexec[k], graph, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();
      cudaGraphExecDestroy(c->gexec[k]);
      c->gexec[k] = nullptr;
    }
  }
  if (!updated) e = cudaGraphInstantiate(&c->gexec[k], graph, 0);
  cudaGraphDestroy(graph);
  if (int rc = cuda_check(c, e, "graph instantiate")) return rc;
  c->g_Q[k] = Q;
  c->g_dt[k] = dt;
  c->g_mu[k] = c->mu;
  c->g_out[k] = copy_out;
  return DGHGKS_OK;
}

int dghgks_steps(dghgks_ctx* c, double* Q, double dt, int nsteps, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q || nsteps < 0) return fail(c, DGHGKS_EARG, "bad argument");
  if (!(dt > 0)) return fail(c, DGHGKS_EARG, "dt must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!c->cap_stream)
    if (int rc = cuda_check(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream"))
      return rc;
  // FP32-mixed contexts: the first step rounds the state into the FP32 copy;
  // every step's update writes it for the next one, which reads it
  const bool copy = c->Qf && nsteps > 1;
  if (c->prof) {  // profiling: the same launches enqueued directly, each recorded
    for (int n = 0; n < nsteps; ++n) enqueue_step(c, Q, dt, s, nullptr, copy && n > 0, copy);
    return after_launch(c, "step launch");
  }
  if (nsteps > 0)
    if (int rc = ensure_graph(c, 0, Q, dt, copy)) return rc;
  if (copy)
    if (int rc = ensure_graph(c, 1, Q, dt, true)) return rc;
  for (int n = 0; n < nsteps; ++n)
    if (int rc = cuda_check(c, cudaGraphLaunch(c->gexec[copy && n > 0 ? 1 : 0], s), "graph launch")) return rc;
  c->launches += 8 * (int64_t)nsteps + (c->Qf && nsteps > 0 ? 1 : 0);  // + the rounding into the copy
  return DGHGKS_OK;
}

int dghgks_totals(dghgks_ctx* c, const double* Q, double* out, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q || !out) return fail(c, DGHGKS_EARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const MeshDev m = mesh_dev(c);
  switch (c->nm) {
    case 4: k_totals_part<4><<<kRedBlocks, RED_THREADS, 0, s>>>(Q, m, c->part); break;
    case 10: k_totals_part<10><<<kRedBlocks, RED_THREADS, 0, s>>>(Q, m, c->part); break;
    default: k_totals_part<20><<<kRedBlocks, RED_THREADS, 0, s>>>(Q, m, c->part); break;
  }
  k_reduce_final<5><<<1, RED_THREADS, 0, s>>>(c->part, kRedBlocks, vol_scale(c), c->red);
  c->launches += 2;
  if (int rc = after_launch(c, "totals launch")) return rc;
  if (int rc = cuda_check(c, cudaMemcpyAsync(c->red_host, c->red, 5 * sizeof(double), cudaMemcpyDeviceToHost, s),
                          "totals copy"))
    return rc;
  if (int rc = cuda_check(c, cudaStreamSynchronize(s), "totals sync")) return rc;
  memcpy(out, c->red_host, 5 * sizeof(double));
  return DGHGKS_OK;
}

static int enqueue_ek(dghgks_ctx* c, const double* Q, double rho0, double* dst_dev, cudaStream_t s) {
  c->ops->ek(c, Q, s);
  k_reduce_final<1><<<1, RED_THREADS, 0, s>>>(c->part, kRedBlocks, vol_scale(c) / (rho0 * c->omega), dst_dev);
  c->launches += 1;
  return after_launch(c, "kinetic energy launch");
}

int dghgks_kinetic_energy(dghgks_ctx* c, const double* Q, double rho0, double* Ek, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q || !Ek) return fail(c, DGHGKS_EARG, "NULL argument");
  if (!(rho0 > 0)) return fail(c, DGHGKS_EARG, "rho0 must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = enqueue_ek(c, Q, rho0, c->red, s)) return rc;
  if (int rc = cuda_check(c, cudaMemcpyAsync(c->red_host, c->red, sizeof(double), cudaMemcpyDeviceToHost, s),
                          "E_k copy"))
    return rc;
  if (int rc = cuda_check(c, cudaStreamSynchronize(s), "E_k sync")) return rc;
  *Ek = c->red_host[0];
  return DGHGKS_OK;
}

int dghgks_enstrophy_dissipation(dghgks_ctx* c, const double* Q, double rho0, double* eps, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q || !eps) return fail(c, DGHGKS_EARG, "NULL argument");
  if (!(rho0 > 0)) return fail(c, DGHGKS_EARG, "rho0 must be > 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->ops->enstrophy(c, Q, s);
  k_reduce_final<1><<<1, RED_THREADS, 0, s>>>(c->part, kRedBlocks, 2.0 * c->mu * vol_scale(c) / (rho0 * c->omega),
                                              c->red);
  c->launches += 1;
  if (int rc = after_launch(c, "enstrophy launch")) return rc;
  if (int rc = cuda_check(c, cudaMemcpyAsync(c->red_host, c->red, sizeof(double), cudaMemcpyDeviceToHost, s),
                          "enstrophy copy"))
    return rc;
  if (int rc = cuda_check(c, cudaStreamSynchronize(s), "enstrophy sync")) return rc;
  *eps = c->red_host[0];
  return DGHGKS_OK;
}

int dghgks_l2_diff(dghgks_ctx* c, const double* A, const double* B, int var, double* out, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!A || !B || !out || var < 0 || var > 4) return fail(c, DGHGKS_EARG, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const MeshDev m = mesh_dev(c);
  switch (c->nm) {
    case 4: k_l2diff_part<4><<<kRedBlocks, RED_THREADS, 0, s>>>(A, B, var, m, c->part); break;
    case 10: k_l2diff_part<10><<<kRedBlocks, RED_THREADS, 0, s>>>(A, B, var, m, c->part); break;
    default: k_l2diff_part<20><<<kRedBlocks, RED_THREADS, 0, s>>>(A, B, var, m, c->part); break;
  }
  k_reduce_final<1><<<1, RED_THREADS, 0, s>>>(c->part, kRedBlocks, vol_scale(c), c->red);
  c->launches += 2;
  if (int rc = after_launch(c, "l2 diff launch")) return rc;
  if (int rc = cuda_check(c, cudaMemcpyAsync(c->red_host, c->red, sizeof(double), cudaMemcpyDeviceToHost, s),
                          "l2 copy"))
    return rc;
  if (int rc = cuda_check(c, cudaStreamSynchronize(s), "l2 sync")) return rc;
  *out = sqrt(c->red_host[0]);
  return DGHGKS_OK;
}

int dghgks_run_host(dghgks_ctx* c, double* Q_host, double dt, int nsteps, double rho0, double* ek_host,
                    void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q_host || nsteps < 0 || !(dt > 0) || !(rho0 > 0)) return fail(c, DGHGKS_EARG, "bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t state = sizeof(double) * 5 * (size_t)c->nm * c->ncell;
  if (!c->Qdev)
    if (int rc = cuda_check(c, cudaMalloc(&c->Qdev, state), "cudaMalloc(run state)")) return rc;
  if (int rc = cuda_check(c, cudaMemcpyAsync(c->Qdev, Q_host, state, cudaMemcpyHostToDevice, s), "H2D state"))
    return rc;
  // E_k of step n runs on a second stream while step n+1 computes: both only
  // read Q^{n+1} until step n+1's stage-2 cell kernel, which waits for it.
  if (ek_host && !c->ek_stream) {
    int rc = cuda_check(c, cudaStreamCreateWithFlags(&c->ek_stream, cudaStreamNonBlocking), "E_k stream");
    if (!rc) rc = cuda_check(c, cudaEventCreateWithFlags(&c->ev_q, cudaEventDisableTiming), "event");
    if (!rc) rc = cuda_check(c, cudaEventCreateWithFlags(&c->ev_ek, cudaEventDisableTiming), "event");
    if (rc) return rc;
  }
  bool ek_pending = false;
  for (int n = 0; n < nsteps; ++n) {
    enqueue_step(c, c->Qdev, dt, s, ek_pending ? c->ev_ek : nullptr, n > 0, n + 1 < nsteps);
    if (int rc = after_launch(c, "step launch")) return rc;
    if (ek_host) {
      cudaStream_t e = c->ek_stream;
      if (int rc = cuda_check(c, cudaEventRecord(c->ev_q, s), "event")) return rc;
      if (int rc = cuda_check(c, cudaStreamWaitEvent(e, c->ev_q, 0), "event")) return rc;
      if (int rc = enqueue_ek(c, c->Qdev, rho0, c->red + (n % 8), e)) return rc;
      if (int rc = cuda_check(c, cudaMemcpyAsync(c->red_host + (n % 8), c->red + (n % 8), sizeof(double),
                                                 cudaMemcpyDeviceToHost, e),
                              "D2H E_k"))
        return rc;
      if (int rc = cuda_check(c, cudaEventRecord(c->ev_ek, e), "event")) return rc;
      ek_pending = true;
      if (n % 8 == 7 || n == nsteps - 1) {
        if (int rc = cuda_check(c, cudaStreamSynchronize(e), "E_k sync")) return rc;
        for (int m = n - (n % 8); m <= n; ++m) ek_host[m] = c->red_host[m % 8];
      }
    }
  }
  if (int rc = cuda_check(c, cudaMemcpyAsync(Q_host, c->Qdev, state, cudaMemcpyDeviceToHost, s), "D2H state"))
    return rc;
  return read_flag(c, s);
}

int dghgks_profile(dghgks_ctx* c, int enable) {
  if (!c) return DGHGKS_EARG;
  if (enable && !c->prof_ev) {
    c->prof_ev = new (std::nothrow) cudaEvent_t[2 * kProfMax];
    c->prof_kind = new (std::nothrow) int[kProfMax];
    if (!c->prof_ev || !c->prof_kind) return fail(c, DGHGKS_ENOMEM, "profile buffers");
    for (int e = 0; e < 2 * kProfMax; ++e)
      if (int rc = cuda_check(c, cudaEventCreate(&c->prof_ev[e]), "cudaEventCreate")) return rc;
  }
  c->prof = enable != 0;
  if (enable) c->prof_n = 0;
  return DGHGKS_OK;
}

int dghgks_profile_read(dghgks_ctx* c, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return DGHGKS_EARG;
  for (int k = 0; k < DGHGKS_NKINDS; ++k) {
    ms[k] = 0;
    launches[k] = 0;
  }
  for (int i = 0; i < c->prof_n; ++i) {
    if (int rc = cuda_check(c, cudaEventSynchronize(c->prof_ev[2 * i + 1]), "event sync")) return rc;
    float t = 0;
    if (int rc = cuda_check(c, cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]), "elapsed"))
      return rc;
    ms[c->prof_kind[i]] += t;
    launches[c->prof_kind[i]] += 1;
  }
  return DGHGKS_OK;
}

static int adj_prepare(dghgks_ctx* c) {
  if (c->precision != DGHGKS_FP64) return fail(c, DGHGKS_EUNSUP, "the adjoint needs an FP64 context");
  if (c->order > 3) return fail(c, DGHGKS_EUNSUP, "the adjoint supports orders 1 to 3");
  if (c->adjH) return DGHGKS_OK;
  const size_t nc = (size_t)c->ncell;
  const size_t state = sizeof(double) * 5 * (size_t)c->nm * nc;
  const size_t fblocks = (size_t)adjoint_face_ctas(c->order, c->n[0], c->n[1], c->n[2]);
  const size_t cblocks = (size_t)((c->n[0] + 3) / 4) * c->n[1] * c->n[2];  // cell CTAs own >= 4 cells
  c->adjMuN = 3 * fblocks + cblocks;
  int rc = cuda_check(c, adjoint_set_attrs(c->order, c->nq), "adjoint attributes");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->adjH, 6 * state), "cudaMalloc(face cotangents)");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->adjLam, state), "cudaMalloc(adjoint state)");
  if (!rc) rc = cuda_check(c, cudaMalloc(&c->adjMu, sizeof(double) * c->adjMuN), "cudaMalloc(adjoint partials)");
  if (rc) {
    cudaFree(c->adjH);
    cudaFree(c->adjLam);
    cudaFree(c->adjMu);
    c->adjH = c->adjLam = c->adjMu = nullptr;
  }
  return rc;
}

// one residual VJP with the viscosity cotangent added to *dmu
static int adj_vjp(dghgks_ctx* c, const double* Q, double dt, AdjIO io, double* dmu, cudaStream_t s) {
  io.H = c->adjH;
  io.mu_part = c->adjMu;
  if (int rc = cuda_check(c, cudaMemsetAsync(c->adjMu, 0, sizeof(double) * c->adjMuN, s), "memset")) return rc;
  adjoint_vjp(c->order, c->nq, Q, gas_par<double>(c, dt), mesh_dev(c), io, s);
  adjoint_mu_sum(c->adjMu, (long long)c->adjMuN, dmu, s);
  c->launches += kAdjointLaunches + 1;
  return after_launch(c, "adjoint launch");
}

int dghgks_residual_vjp(dghgks_ctx* c, const double* Q, double dt, const double* lamL, const double* lamLt,
                        double* lamQ, double* dmu, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Q || !lamL || !lamLt || !lamQ || !dmu) return fail(c, DGHGKS_EARG, "NULL argument");
  if (!(dt > 0)) return fail(c, DGHGKS_EARG, "dt must be > 0");
  if (lamQ == Q || lamQ == lamL || lamQ == lamLt) return fail(c, DGHGKS_EARG, "lamQ must not alias the inputs");
  if (int rc = adj_prepare(c)) return rc;
  AdjIO io{};
  io.lamA = lamL;
  io.lamB = lamLt;
  io.cLA = 1.0;
  io.cLB = 0.0;
  io.cTA = 0.0;
  io.cTB = 1.0;
  io.out = lamQ;
  return adj_vjp(c, Q, dt, io, dmu, static_cast<cudaStream_t>(stream));
}

int dghgks_adjoint_step(dghgks_ctx* c, const double* Qn, const double* lam_next, double dt, double* lam_n,
                        double* dJ_dmu, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (!Qn || !lam_next || !lam_n || !dJ_dmu) return fail(c, DGHGKS_EARG, "NULL argument");
  if (!(dt > 0)) return fail(c, DGHGKS_EARG, "dt must be > 0");
  if (lam_n == Qn) return fail(c, DGHGKS_EARG, "lam_n must not alias Qn");
  if (int rc = adj_prepare(c)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // recompute Q* from the checkpoint (one forward stage)
  c->ops->faces(c, Qn, FACES_FP64, dt, s);
  c->ops->cell(c, MODE_STAGE1, const_cast<double*>(Qn), nullptr, nullptr, dt, s, false, false);
  const double* Qs = static_cast<const double*>(c->Qs);
  // stage 2 at Q*: only L_t(Q*) enters Q^{n+1}, with dt^2/3
  AdjIO io2{};
  io2.lamA = lam_next;
  io2.cTA = dt * dt / 3.0;
  io2.out = c->adjLam;
  if (int rc = adj_vjp(c, Qs, dt, io2, dJ_dmu, s)) return rc;
  // stage 1 at Q^n: L with dt (direct) and dt/2 (through Q*), L_t with dt^2/6 and dt^2/8
  AdjIO io1{};
  io1.lamA = lam_next;
  io1.lamB = c->adjLam;
  io1.cLA = dt;
  io1.cLB = 0.5 * dt;
  io1.cTA = dt * dt / 6.0;
  io1.cTB = dt * dt / 8.0;
  io1.out = lam_n;
  io1.addA = lam_next;
  io1.addB = c->adjLam;
  return adj_vjp(c, Qn, dt, io1, dJ_dmu, s);
}

int dghgks_kinetic_energy_vjp(dghgks_ctx* c, const double* Q, double rho0, double* dEk_dQ, void* stream) {
  if (!c) return DGHGKS_EARG;
  if (c->order > 3) return fail(c, DGHGKS_EUNSUP, "the adjoint supports orders 1 to 3");
  if (!Q || !dEk_dQ || dEk_dQ == Q) return fail(c, DGHGKS_EARG, "bad argument");
  if (!(rho0 > 0)) return fail(c, DGHGKS_EARG, "rho0 must be > 0");
  adjoint_ek_vjp(c->order, c->nq, Q, mesh_dev(c), vol_scale(c) / (rho0 * c->omega), dEk_dQ,
                 static_cast<cudaStream_t>(stream));
  c->launches += 1;
  return after_launch(c, "E_k VJP launch");
}

int dghgks_status(dghgks_ctx* c, void* stream) {
  if (!c) return DGHGKS_EARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int rc = cuda_check(c, cudaGetLastError(), "pending error")) return rc;
  return read_flag(c, s);
}

}  // extern "C"
