// DG-HGKS residual kernels (Sec. 3 of arXiv:2202.13821, Eqs. operator,
// surface, volume, two-stage), templated on the flux arithmetic R (double,
// or float in the FP32-mixed path), the degree ORDER and the Gauss count NQ.
//
// One stage = 3 face launches (one per normal direction) + 1 cell launch:
//
//   k_face<D>: a CTA owns FB consecutive faces along x normal to axis D.  It
//     stages the modal coefficients of the two cells of each face in shared
//     memory, evaluates Q_h and grad Q_h on both sides of its NQ^2 Gauss
//     points (one warp per point, lanes over faces), computes F_b and
//     d_t F_b there (Eq. flux, local frame with the normal first), and
//     projects w |Gamma| F onto the NT tangential Legendre products of the
//     face.  Only those face moments G reach HBM (10 x NT values per face);
//     point values never do.
//
//   k_cell<MODE>: a CTA owns CB consecutive cells along x, one thread per
//     (cell, Gauss point).  It evaluates the interior flux of Eq. (flux-2)
//     at the NQ^3 points, projects w |K| F . grad B_n in shared memory, adds
//     the six faces' moments with the sign and parity of Eq. (operator)
//     (the cell is right of its low face: +(-1)^{n_D} G, left of its high
//     face: -G), multiplies by the diagonal inverse mass matrix, and applies
//     the epilogue:
//       MODE 0: write L = M^-1 R and L_t = M^-1 R_t
//       MODE 1: Q* = Q^n + dt/2 L + dt^2/8 L_t, Acc = Q^n + dt L + dt^2/6 L_t
//       MODE 2: Q^{n+1} = Acc + dt^2/3 L_t(Q*)
//     The stage arithmetic is always FP64.
//
// Each face is computed exactly once and written by exactly one CTA, and
// every residual coefficient is summed in a fixed order: results are
// bit-reproducible from run to run (no floating-point atomics).
// A non-physical state (rho <= 0 or p <= 0) sets bit 0 of *flag.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_tables.cuh"
#include "gks_point.cuh"

namespace dghgks {

struct MeshDev {
  int nx, ny, nz;
  long long ncell;
  double h[3];
  double vol;
};

constexpr int FB = 32;  // faces per CTA in k_face

template <int NQ>
struct CellTile {
  static constexpr int CB = NQ == 1 ? 32 : NQ == 2 ? 16 : NQ == 3 ? 8 : NQ == 4 ? 4 : 2;
};

template <class R, int ORDER, int NQ>
struct FaceSmem {
  static constexpr int NM = n_modes(ORDER), NT = n_tmodes(ORDER), NP = NQ * NQ, NC = 5 * NM;
  static constexpr size_t coef = sizeof(R) * NC * FB;  // one side
  static constexpr size_t fs = sizeof(R) * 10 * NP * FB;
  static constexpr size_t phi = sizeof(R) * NT * NP;
  static constexpr size_t bytes = 2 * coef + fs + phi;
};

template <class R, int ORDER, int NQ>
struct CellSmem {
  static constexpr int NM = n_modes(ORDER), NP = NQ * NQ * NQ, NC = 5 * NM, CB = CellTile<NQ>::CB;
  static constexpr size_t coef = sizeof(R) * NC * CB;
  static constexpr size_t fs = sizeof(R) * 30 * NP * CB;
  static constexpr size_t db = sizeof(R) * NM * NP * 3;
  static constexpr size_t tabs = sizeof(double) * NM + sizeof(int) * 6 * NM;
  static constexpr size_t bytes = coef + fs + db + tabs;
};

__device__ __forceinline__ int wrapm(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------------------
// Face kernel
// ---------------------------------------------------------------------------
template <class R, int ORDER, int NQ, int D>
__global__ void __launch_bounds__(FB* NQ* NQ)
    k_face(const double* __restrict__ Q, R* __restrict__ G, const GasPar<R> gp, const MeshDev m,
           unsigned* __restrict__ flag) {
  using S = FaceSmem<R, ORDER, NQ>;
  constexpr int NM = S::NM, NT = S::NT, NP = S::NP, NC = S::NC;
  constexpr int T1 = tan1(D), T2 = tan2(D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R(*cL)[FB] = reinterpret_cast<R(*)[FB]>(smem_raw);
  R(*cR)[FB] = reinterpret_cast<R(*)[FB]>(smem_raw + S::coef);
  R(*Fs)[NP][FB] = reinterpret_cast<R(*)[NP][FB]>(smem_raw + 2 * S::coef);
  R(*phi)[NP] = reinterpret_cast<R(*)[NP]>(smem_raw + 2 * S::coef + S::fs);

  const int tid = threadIdx.x;
  const int f = tid % FB, p = tid / FB;
  const int i0 = blockIdx.x * FB, j = blockIdx.y, k = blockIdx.z;
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  const long long nc = m.ncell;

  // stage the coefficients of the left (-e_D) and right cells of each face
  for (int e = tid; e < 2 * NC * FB; e += FB * NP) {
    const int ff = e % FB, rest = e / FB, c = rest % NC, side = rest / NC;
    const int i = i0 + ff;
    R val = R(0);
    if (i < nx) {
      int ci = i, cj = j, ck = k;
      if (side == 0) {
        if (D == 0) ci = wrapm(i - 1, nx);
        if (D == 1) cj = wrapm(j - 1, ny);
        if (D == 2) ck = wrapm(k - 1, nz);
      }
      val = (R)__ldg(Q + (size_t)c * nc + ((size_t)ck * ny + cj) * nx + ci);
    }
    if (side == 0)
      cL[c][ff] = val;
    else
      cR[c][ff] = val;
  }
  for (int e = tid; e < NT * NP; e += FB * NP) {
    const int t = e / NP, pp = e % NP;
    phi[t][pp] = leg<R>(tmode_p(t), (R)gauss_x(NQ, pp / NQ)) * leg<R>(tmode_q(t), (R)gauss_x(NQ, pp % NQ));
  }
  __syncthreads();

  const int i = i0 + f;
  const bool active = i < nx;
  const int a = p / NQ, b = p % NQ;
  const R xa = (R)gauss_x(NQ, a), xb = (R)gauss_x(NQ, b);
  R La[ORDER + 1], dLa[ORDER + 1], Lb[ORDER + 1], dLb[ORDER + 1];
#pragma unroll
  for (int n = 0; n <= ORDER; ++n) {
    La[n] = leg<R>(n, xa);
    dLa[n] = dleg<R>(n, xa);
    Lb[n] = leg<R>(n, xb);
    dLb[n] = dleg<R>(n, xb);
  }
  const R sD = R(2) / (R)m.h[D], s1 = R(2) / (R)m.h[T1], s2 = R(2) / (R)m.h[T2];

  // traces: side 0 at r_D = +1 of the left cell, side 1 at r_D = -1 of the right cell
  R q[2][5], dq[2][3][5];  // dq[side][axis][var], global axes
#pragma unroll
  for (int side = 0; side < 2; ++side) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R s0 = R(0), gD = R(0), g1 = R(0), g2 = R(0);
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) {
        constexpr int dummy = 0;
        (void)dummy;
        const int nD = mode_exp(mm, D), n1 = mode_exp(mm, T1), n2 = mode_exp(mm, T2);
        // P_n(+1) = 1, P_n(-1) = (-1)^n; P'_n(+1) = n(n+1)/2, P'_n(-1) = (-1)^(n+1) n(n+1)/2
        const R pn = (side == 0 || (nD % 2 == 0)) ? R(1) : R(-1);
        const R dpn = R(nD * (nD + 1) / 2) * ((side == 0 || (nD % 2 == 1)) ? R(1) : R(-1));
        const R c = (side == 0) ? cL[v * NM + mm][f] : cR[v * NM + mm][f];
        const R t12 = La[n1] * Lb[n2];
        s0 += c * (pn * t12);
        gD += c * (dpn * t12);
        g1 += c * (pn * dLa[n1] * Lb[n2]);
        g2 += c * (pn * La[n1] * dLb[n2]);
      }
      q[side][v] = s0;
      dq[side][D][v] = gD * sD;
      dq[side][T1][v] = g1 * s1;
      dq[side][T2][v] = g2 * s2;
    }
  }

  // local frame: axes (D, D+1, D+2) cyclic; momentum components alike
  constexpr int A0 = D, A1 = (D + 1) % 3, A2 = (D + 2) % 3;
  R ql[5], qr[5], dql[3][5], dqr[3][5];
  {
    const int ax[3] = {A0, A1, A2};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      R* qq = side == 0 ? ql : qr;
      qq[0] = q[side][0];
      qq[1] = q[side][1 + A0];
      qq[2] = q[side][1 + A1];
      qq[3] = q[side][1 + A2];
      qq[4] = q[side][4];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) {
        R* dd = side == 0 ? dql[ii] : dqr[ii];
        const R* src = dq[side][ax[ii]];
        dd[0] = src[0];
        dd[1] = src[1 + A0];
        dd[2] = src[1 + A1];
        dd[3] = src[1 + A2];
        dd[4] = src[4];
      }
    }
  }
  R Fl[5], Ftl[5];
  const bool ok = iface_flux(ql, dql, qr, dqr, gp, Fl, Ftl);
  if (active && !ok) atomicOr(flag, 1u);
  const R w = active ? (R)(gauss_w(NQ, a) * gauss_w(NQ, b) * (m.vol / m.h[D])) : R(0);
  Fs[0][p][f] = w * Fl[0];
  Fs[1 + A0][p][f] = w * Fl[1];
  Fs[1 + A1][p][f] = w * Fl[2];
  Fs[1 + A2][p][f] = w * Fl[3];
  Fs[4][p][f] = w * Fl[4];
  Fs[5][p][f] = w * Ftl[0];
  Fs[6 + A0][p][f] = w * Ftl[1];
  Fs[6 + A1][p][f] = w * Ftl[2];
  Fs[6 + A2][p][f] = w * Ftl[3];
  Fs[9][p][f] = w * Ftl[4];
  __syncthreads();

  // tangential projection: G[D][c][t][face] = sum_p Fs[c][p] phi_t(p)
  if (active) {
    const size_t face = ((size_t)k * ny + j) * nx + i;
    for (int o = p; o < 10 * NT; o += NP) {
      const int c = o / NT, t = o % NT;
      R s = R(0);
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) s += Fs[c][pp][f] * phi[t][pp];
      G[((size_t)(D * 10 + c) * NT + t) * nc + face] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Cell kernel
// ---------------------------------------------------------------------------
enum { MODE_RESIDUAL = 0, MODE_STAGE1 = 1, MODE_STAGE2 = 2 };

template <class R, int ORDER, int NQ, int MODE>
__global__ void __launch_bounds__(CellTile<NQ>::CB* NQ* NQ* NQ)
    k_cell(const double* __restrict__ Qin, const R* __restrict__ G, double* __restrict__ out0,
           double* __restrict__ out1, const double* __restrict__ acc, const GasPar<R> gp, const MeshDev m,
           const double dt, unsigned* __restrict__ flag) {
  using S = CellSmem<R, ORDER, NQ>;
  constexpr int NM = S::NM, NP = S::NP, NC = S::NC, CB = S::CB, NT = n_tmodes(ORDER);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R(*coef)[CB] = reinterpret_cast<R(*)[CB]>(smem_raw);
  R(*Fs)[NP][CB] = reinterpret_cast<R(*)[NP][CB]>(smem_raw + S::coef);
  R(*dB)[NP][3] = reinterpret_cast<R(*)[NP][3]>(smem_raw + S::coef + S::fs);
  double* invM = reinterpret_cast<double*>(smem_raw + S::coef + S::fs + S::db);
  int* tix = reinterpret_cast<int*>(invM + NM);  // [3][NM] tangential index, then [3][NM] parity sign

  const int tid = threadIdx.x, nthr = CB * NP;
  const int c = tid % CB, p = tid / CB;
  const int i0 = blockIdx.x * CB, j = blockIdx.y, k = blockIdx.z;
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  const long long nc = m.ncell;
  const size_t row = ((size_t)k * ny + j) * nx;

  for (int e = tid; e < NC * CB; e += nthr) {
    const int cc = e % CB, comp = e / CB, i = i0 + cc;
    coef[comp][cc] = (i < nx) ? (R)__ldg(Qin + (size_t)comp * nc + row + i) : R(0);
  }
  for (int e = tid; e < NM * NP * 3; e += nthr) {
    const int d = e % 3, pp = (e / 3) % NP, mm = e / (3 * NP);
    const int pa[3] = {pp / (NQ * NQ), (pp / NQ) % NQ, pp % NQ};
    R v = R(1);
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      const R x = (R)gauss_x(NQ, pa[dd]);
      const int n = mode_exp(mm, dd);
      v *= (dd == d) ? dleg<R>(n, x) : leg<R>(n, x);
    }
    dB[mm][pp][d] = v;
  }
  for (int e = tid; e < NM; e += nthr) {
    invM[e] = (double)((2 * mode_exp(e, 0) + 1) * (2 * mode_exp(e, 1) + 1) * (2 * mode_exp(e, 2) + 1)) / m.vol;
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      tix[D * NM + e] = tmode_index(mode_exp(e, tan1(D)), mode_exp(e, tan2(D)));
      tix[3 * NM + D * NM + e] = (mode_exp(e, D) % 2 == 0) ? 1 : -1;
    }
  }
  __syncthreads();

  // interior flux at point p = (a, b, cz) of cell c
  {
    const int i = i0 + c;
    const bool active = i < nx;
    const int pa[3] = {p / (NQ * NQ), (p / NQ) % NQ, p % NQ};
    R L1[3][ORDER + 1], dL1[3][ORDER + 1];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R x = (R)gauss_x(NQ, pa[d]);
#pragma unroll
      for (int n = 0; n <= ORDER; ++n) {
        L1[d][n] = leg<R>(n, x);
        dL1[d][n] = dleg<R>(n, x);
      }
    }
    const R sc[3] = {R(2) / (R)m.h[0], R(2) / (R)m.h[1], R(2) / (R)m.h[2]};
    R q[5], dq[3][5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R s0 = R(0), g0 = R(0), g1 = R(0), g2 = R(0);
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) {
        const int e0 = mode_exp(mm, 0), e1 = mode_exp(mm, 1), e2 = mode_exp(mm, 2);
        const R cv = coef[v * NM + mm][c];
        s0 += cv * (L1[0][e0] * L1[1][e1] * L1[2][e2]);
        g0 += cv * (dL1[0][e0] * L1[1][e1] * L1[2][e2]);
        g1 += cv * (L1[0][e0] * dL1[1][e1] * L1[2][e2]);
        g2 += cv * (L1[0][e0] * L1[1][e1] * dL1[2][e2]);
      }
      q[v] = s0;
      dq[0][v] = g0 * sc[0];
      dq[1][v] = g1 * sc[1];
      dq[2][v] = g2 * sc[2];
    }
    R F[3][5], Ft[3][5];
    const bool ok = interior_flux(q, dq, gp, F, Ft);
    if (active && !ok) atomicOr(flag, 1u);
    const R w = active ? (R)(gauss_w(NQ, pa[0]) * gauss_w(NQ, pa[1]) * gauss_w(NQ, pa[2]) * m.vol) : R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R wd = w * sc[d];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Fs[d * 5 + v][p][c] = wd * F[d][v];
        Fs[15 + d * 5 + v][p][c] = wd * Ft[d][v];
      }
    }
  }
  __syncthreads();

  // projection, face assembly, inverse mass matrix, stage epilogue
  for (int o = tid; o < CB * NC; o += nthr) {
    const int cc = o % CB, rest = o / CB, mm = rest % NM, v = rest / NM;
    const int i = i0 + cc;
    if (i >= nx) continue;
    R sF = R(0), sT = R(0);
    for (int pp = 0; pp < NP; ++pp) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R bb = dB[mm][pp][d];
        sF += Fs[d * 5 + v][pp][cc] * bb;
        sT += Fs[15 + d * 5 + v][pp][cc] * bb;
      }
    }
    const size_t cell = row + i;
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      const int t = tix[D * NM + mm];
      const R sg = (R)tix[3 * NM + D * NM + mm];
      size_t up;
      if (D == 0)
        up = row + wrapm(i + 1, nx);
      else if (D == 1)
        up = ((size_t)k * ny + wrapm(j + 1, ny)) * nx + i;
      else
        up = ((size_t)wrapm(k + 1, nz) * ny + j) * nx + i;
      const R* gF = G + ((size_t)(D * 10 + v) * NT + t) * nc;
      const R* gT = G + ((size_t)(D * 10 + 5 + v) * NT + t) * nc;
      sF += sg * gF[cell] - gF[up];
      sT += sg * gT[cell] - gT[up];
    }
    const double Lv = (double)sF * invM[mm], Ltv = (double)sT * invM[mm];
    const size_t idx = (size_t)(v * NM + mm) * nc + cell;
    if (MODE == MODE_RESIDUAL) {
      out0[idx] = Lv;
      out1[idx] = Ltv;
    } else if (MODE == MODE_STAGE1) {
      const double qn = Qin[idx];
      out0[idx] = qn + 0.5 * dt * Lv + (dt * dt / 8.0) * Ltv;
      out1[idx] = qn + dt * Lv + (dt * dt / 6.0) * Ltv;
    } else {
      out0[idx] = acc[idx] + (dt * dt / 3.0) * Ltv;
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 reductions (deterministic two-pass): conserved totals and E_k
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&acc)[NV], double* __restrict__ part) {
  __shared__ double sh[NV][RED_THREADS];
#pragma unroll
  for (int v = 0; v < NV; ++v) sh[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int v = 0; v < NV; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) part[(size_t)blockIdx.x * NV + v] = sh[v][0];
}

template <int NM>
__global__ void __launch_bounds__(RED_THREADS) k_totals_part(const double* __restrict__ Q, long long nc,
                                                             double* __restrict__ part) {
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < nc; c += (long long)gridDim.x * RED_THREADS)
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += Q[(size_t)(v * NM) * nc + c];
  block_reduce_store<5>(acc, part);
}

template <int ORDER, int NQ>
__global__ void __launch_bounds__(RED_THREADS) k_ek_part(const double* __restrict__ Q, long long nc,
                                                         double* __restrict__ part) {
  constexpr int NM = n_modes(ORDER);
  double acc[1] = {0};
  for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < nc; c += (long long)gridDim.x * RED_THREADS) {
    double co[4][NM];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) co[v][mm] = Q[(size_t)(v * NM + mm) * nc + c];
#pragma unroll
    for (int a = 0; a < NQ; ++a)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int cz = 0; cz < NQ; ++cz) {
          double qv[4] = {0, 0, 0, 0};
#pragma unroll
          for (int mm = 0; mm < NM; ++mm) {
            const double B = leg<double>(mode_exp(mm, 0), gauss_x(NQ, a)) * leg<double>(mode_exp(mm, 1), gauss_x(NQ, b)) *
                             leg<double>(mode_exp(mm, 2), gauss_x(NQ, cz));
#pragma unroll
            for (int v = 0; v < 4; ++v) qv[v] += co[v][mm] * B;
          }
          acc[0] += gauss_w(NQ, a) * gauss_w(NQ, b) * gauss_w(NQ, cz) * 0.5 *
                    (qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]) / qv[0];
        }
  }
  block_reduce_store<1>(acc, part);
}

template <int NV>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double* __restrict__ part, int nblocks,
                                                              double scale, double* __restrict__ out) {
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0;
  for (int b = threadIdx.x; b < nblocks; b += RED_THREADS)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] += part[(size_t)b * NV + v];
  __shared__ double sh[NV][RED_THREADS];
#pragma unroll
  for (int v = 0; v < NV; ++v) sh[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int v = 0; v < NV; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = sh[v][0] * scale;
}

}  // namespace dghgks
