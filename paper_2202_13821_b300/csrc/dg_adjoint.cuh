// Reverse-mode (adjoint) kernels of the DG-HGKS residual, FP64.
//
// The residual of Sec. 3 (Eq. operator) is a linear projection of point
// fluxes, which are nonlinear functions of the traces, which are linear in
// the modal coefficients:
//   Q --trace--> (q, grad q)(x_m) --flux (Eq. flux / flux-2)--> F(x_m)
//     --projection (Eqs. surface, volume)--> R --M^-1--> L.
// Given cotangents of (L, L_t) the vector-Jacobian product runs backwards:
//   mu = M^-1 lambda (diagonal); the projection transposed gives the
//   cotangent of F and F_t at every Gauss point; the point-flux Jacobian
//   transposed gives the cotangents of the traces and of the viscosity; the
//   trace transposed gives the cotangent of Q.
// The point-flux Jacobian-transpose products are the hand-written reverse
// mode of gks_point_adj.cuh: one backward sweep per Gauss point, after
// recomputing the point's forward intermediates.  Exact to rounding; every
// sum is taken in a fixed order.
#pragma once
#include <cmath>

#include "adjoint.h"
#include "dg_kernels.cuh"
#include "gks_point_adj.cuh"

namespace dghgks {

// faces per CTA of the face VJP: 32, or 16 for P3 (its shared-memory staging
// of both cells' coefficients and cotangents would not fit 227 KB at 32)
template <int ORDER>
constexpr int adj_fb() {
  return ORDER >= 3 ? 16 : FB;
}

template <int ORDER, int NQ>
struct FaceAdjSmem {
  static constexpr int FBA = adj_fb<ORDER>();
  static constexpr int NM = n_modes(ORDER), NP = NQ * NQ, NC = 5 * NM;
  static constexpr size_t coef = sizeof(double) * NC * FBA;  // one side, one array
  static constexpr size_t g = sizeof(double) * 40 * NP * FBA;
  static constexpr size_t red = sizeof(double) * FBA * NP;
  static constexpr size_t bytes = 2 * coef + 4 * coef + g + red + sizeof(double) * NM;
};

// cotangent scale of mode n: lambda_R = M^-1 lambda_L with M^-1 = prod(2 n_d + 1) / |K|
DG_HD double inv_mass(int mm, double vol) {
  return (double)((2 * mode_exp(mm, 0) + 1) * (2 * mode_exp(mm, 1) + 1) * (2 * mode_exp(mm, 2) + 1)) / vol;
}

// ---------------------------------------------------------------------------
// Face VJP: H[D][side][comp][face] = sum over the face's Gauss points of the
// trace transpose of the traces' cotangents; mu_part[block] = viscosity part.
// FTO: the cotangent of L is zero (io.cLA = io.cLB = 0: stage 2 of the S2O4
// adjoint), so the point sweeps differentiate F_t alone.
// ---------------------------------------------------------------------------
template <int ORDER, int NQ, int D, bool FTO = false>
__global__ void __launch_bounds__(adj_fb<ORDER>() * NQ * NQ)
    k_face_vjp(const double* __restrict__ Q, const GasPar<double> gp, const MeshDev m, const AdjIO io,
               const size_t mu_offset) {
  using S = FaceAdjSmem<ORDER, NQ>;
  constexpr int FBA = S::FBA;
  constexpr int NM = S::NM, NP = S::NP, NC = S::NC;
  constexpr int T1 = tan1(D), T2 = tan2(D);
  constexpr int A0 = D, A1 = (D + 1) % 3, A2 = (D + 2) % 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double(*cq)[NC][FBA] = reinterpret_cast<double(*)[NC][FBA]>(smem_raw);                  // [side]
  double(*cmu)[NC][FBA] = reinterpret_cast<double(*)[NC][FBA]>(smem_raw + 2 * S::coef);   // [side*2 + kind]
  double(*gs)[NP][FBA] = reinterpret_cast<double(*)[NP][FBA]>(smem_raw + 6 * S::coef);   // [input][point]
  double(*red)[FBA] = reinterpret_cast<double(*)[FBA]>(smem_raw + 6 * S::coef + S::g);  // [point]

  const int tid = threadIdx.x, nthr = FBA * NP;
  const int f = tid % FBA, p = tid / FBA;
  const int i0 = blockIdx.x * FBA, j = blockIdx.y, k = blockIdx.z;
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  const long long nc = m.ncell;

  // stage Q and the mass-scaled cotangents of both cells of each face
  for (int e = tid; e < 2 * NC * FBA; e += nthr) {
    const int ff = e % FBA, rest = e / FBA, c = rest % NC, side = rest / NC;
    const int i = i0 + ff;
    double q = 0, mR = 0, mT = 0;
    if (i < nx) {
      int ci = i, cj = j, ck = k;
      if (side == 0) {
        if (D == 0) ci = wrapm(i - 1, nx);
        if (D == 1) cj = wrapm(j - 1, ny);
        if (D == 2) ck = wrapm(k - 1, nz);
      }
      const size_t idx = (size_t)c * nc + ((size_t)ck * ny + cj) * nx + ci;
      const double iM = inv_mass(c % NM, cell_vol64(m, ci, cj, ck));
      const double a = io.lamA[idx], b = io.lamB ? io.lamB[idx] : 0.0;
      q = Q[idx];
      mR = iM * (io.cLA * a + io.cLB * b);
      mT = iM * (io.cTA * a + io.cTB * b);
    }
    cq[side][c][ff] = q;
    if (!FTO) cmu[side * 2][c][ff] = mR;
    cmu[side * 2 + 1][c][ff] = mT;
  }
  __syncthreads();

  const int i = i0 + f;
  const bool active = i < nx;
  const int a = p / NQ, b = p % NQ;
  const double xa = gauss_x(NQ, a), xb = gauss_x(NQ, b);
  double La[ORDER + 1], dLa[ORDER + 1], Lb[ORDER + 1], dLb[ORDER + 1];
#pragma unroll
  for (int n = 0; n <= ORDER; ++n) {
    La[n] = leg<double>(n, xa);
    dLa[n] = dleg<double>(n, xa);
    Lb[n] = leg<double>(n, xb);
    dLb[n] = dleg<double>(n, xb);
  }
  // gradient scales: along D those of the left and right cells, tangential
  // ones shared by both cells (rectilinear mesh); the face area
  const int cidx[3] = {active ? i : 0, j, k};
  const int nAx = D == 0 ? nx : (D == 1 ? ny : nz);
  const double sDs[2] = {cell_sc<double>(m, D, wrapm(cidx[D] - 1, nAx)), cell_sc<double>(m, D, cidx[D])};
  const double s1 = cell_sc<double>(m, T1, cidx[T1]), s2 = cell_sc<double>(m, T2, cidx[T2]);
  const double w = active ? gauss_w(NQ, a) * gauss_w(NQ, b) * face_area<double>(m, D, cidx[T1], cidx[T2]) : 0.0;

  // traces (global axes) and the flux cotangents of the point
  double q[2][5], dq[2][3][5], lF[5], lT[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    lF[v] = 0.0;
    lT[v] = 0.0;
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    // the face adds -w F B^L to the left cell and +w F B^R to the right cell
    const double sg = side == 0 ? -w : w;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double s0 = 0, gD = 0, g1 = 0, g2 = 0;
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) {
        const int nD = mode_exp(mm, D), n1 = mode_exp(mm, T1), n2 = mode_exp(mm, T2);
        const double pn = (side == 0 || (nD % 2 == 0)) ? 1.0 : -1.0;
        const double dpn = (double)(nD * (nD + 1) / 2) * ((side == 0 || (nD % 2 == 1)) ? 1.0 : -1.0);
        const double c = cq[side][v * NM + mm][f];
        const double B = pn * La[n1] * Lb[n2];
        s0 += c * B;
        gD += c * (dpn * La[n1] * Lb[n2]);
        g1 += c * (pn * dLa[n1] * Lb[n2]);
        g2 += c * (pn * La[n1] * dLb[n2]);
        if (!FTO) lF[v] += sg * B * cmu[side * 2][v * NM + mm][f];
        lT[v] += sg * B * cmu[side * 2 + 1][v * NM + mm][f];
      }
      q[side][v] = s0;
      dq[side][D][v] = gD * sDs[side];
      dq[side][T1][v] = g1 * s1;
      dq[side][T2][v] = g2 * s2;
    }
  }

  // Reverse mode of the point flux (gks_point_adj.cuh): the cotangents of
  // F, F_t in the local frame give those of both sides' traces and of mu in
  // one backward sweep.
  double ql0[2][5], dql0[2][3][5];
  {
    const int ax[3] = {A0, A1, A2};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      ql0[side][0] = q[side][0];
      ql0[side][1] = q[side][1 + A0];
      ql0[side][2] = q[side][1 + A1];
      ql0[side][3] = q[side][1 + A2];
      ql0[side][4] = q[side][4];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) {
        dql0[side][ii][0] = dq[side][ax[ii]][0];
        dql0[side][ii][1] = dq[side][ax[ii]][1 + A0];
        dql0[side][ii][2] = dq[side][ax[ii]][1 + A1];
        dql0[side][ii][3] = dq[side][ax[ii]][1 + A2];
        dql0[side][ii][4] = dq[side][ax[ii]][4];
      }
    }
  }
  const double Flb[5] = {lF[0], lF[1 + A0], lF[1 + A1], lF[1 + A2], lF[4]};
  const double Ftlb[5] = {lT[0], lT[1 + A0], lT[1 + A1], lT[1 + A2], lT[4]};
  double qlb[2][5], dqlb[2][3][5], gmu = 0.0;
  iface_flux_vjp<double, FTO>(ql0[0], dql0[0], ql0[1], dql0[1], gp, Flb, Ftlb, qlb[0], dqlb[0], qlb[1], dqlb[1], gmu);
  if (!active) gmu = 0.0;
  // back to global variables and axes: local index of a global momentum component
  const int loc[3] = {(0 - A0 + 3) % 3, (1 - A0 + 3) % 3, (2 - A0 + 3) % 3};
#pragma unroll
  for (int side = 0; side < 2; ++side)
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const int lv = (v >= 1 && v <= 3) ? 1 + loc[v - 1] : v;
      gs[side * 20 + v][p][f] = active ? qlb[side][lv] : 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) gs[side * 20 + 5 + d * 5 + v][p][f] = active ? dqlb[side][loc[d]][lv] : 0.0;
    }
  red[p][f] = gmu;
  __syncthreads();

  // trace transpose, summed over the face's points in a fixed order:
  // H[side][v][n] = sum_p B_n(p) g_q[v] + sum_d (2/h_d) dB_n/dr_d(p) g_dq[d][v]
  if (active) {
    const size_t face = ((size_t)k * ny + j) * nx + i;
    for (int o = p; o < 2 * NC; o += NP) {
      const int side = o / NC, comp = o % NC, v = comp / NM, mm = comp % NM;
      const int nD = mode_exp(mm, D), n1 = mode_exp(mm, T1), n2 = mode_exp(mm, T2);
      const double pn = (side == 0 || (nD % 2 == 0)) ? 1.0 : -1.0;
      const double dpn = (double)(nD * (nD + 1) / 2) * ((side == 0 || (nD % 2 == 1)) ? 1.0 : -1.0);
      double acc = 0.0;
      for (int pp = 0; pp < NP; ++pp) {
        const double xa2 = gauss_x(NQ, pp / NQ), xb2 = gauss_x(NQ, pp % NQ);
        const double l1 = leg<double>(n1, xa2), l2 = leg<double>(n2, xb2);
        const int base = side * 20;
        acc += pn * l1 * l2 * gs[base + v][pp][f];
        acc += sDs[side] * dpn * l1 * l2 * gs[base + 5 + D * 5 + v][pp][f];
        acc += s1 * pn * dleg<double>(n1, xa2) * l2 * gs[base + 5 + T1 * 5 + v][pp][f];
        acc += s2 * pn * l1 * dleg<double>(n2, xb2) * gs[base + 5 + T2 * 5 + v][pp][f];
      }
      io.H[(((size_t)D * 2 + side) * NC + comp) * nc + face] = acc;
    }
  }
  // viscosity cotangent: per-CTA partial in a fixed order
  if (tid == 0) {
    double s = 0.0;
    for (int pp = 0; pp < NP; ++pp)
      for (int ff = 0; ff < FBA; ++ff) s += red[pp][ff];
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    io.mu_part[mu_offset + blk] = s;
  }
}

// ---------------------------------------------------------------------------
// Cell VJP: out = addA + addB + (volume part + the six faces' H) of the cell.
// ---------------------------------------------------------------------------
// (the forward kernel's layout: one lane per Gauss point, a cell over GW
// warps; each warp reduces its points' share, the GW partial sums meet in
// shared memory)
template <int ORDER, int NQ>
struct CellAdjSmem {
  using LY = CellLayout<ORDER, NQ>;
  static constexpr int NM = LY::NM, NC = 5 * NM, CB = LY::CB;
  static constexpr int NOP2 = (NC + LY::PG - 1) / LY::PG * LY::PG;
  static constexpr size_t coef = sizeof(double) * NC * CB;
  static constexpr size_t red = sizeof(double) * CB * LY::GW * NOP2;
  static constexpr size_t bytes = 3 * coef + red + sizeof(double) * LY::WARPS * 32;
};

// (FTO as for the face VJP)
template <int ORDER, int NQ, bool FTO = false>
__global__ void __launch_bounds__(CellLayout<ORDER, NQ>::WARPS * 32)
    k_cell_vjp(const double* __restrict__ Q, const GasPar<double> gp, const MeshDev m, const AdjIO io,
               const size_t mu_offset) {
  using LY = CellLayout<ORDER, NQ>;
  using S = CellAdjSmem<ORDER, NQ>;
  constexpr int NM = LY::NM, NP = LY::NP, NC = S::NC, CB = LY::CB, PG = LY::PG, GW = LY::GW, NOP2 = S::NOP2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double(*cq)[CB] = reinterpret_cast<double(*)[CB]>(smem_raw);
  double(*cmuR)[CB] = reinterpret_cast<double(*)[CB]>(smem_raw + S::coef);
  double(*cmuT)[CB] = reinterpret_cast<double(*)[CB]>(smem_raw + 2 * S::coef);
  double(*red)[GW][NOP2] = reinterpret_cast<double(*)[GW][NOP2]>(smem_raw + 3 * S::coef);
  double* mured = reinterpret_cast<double*>(smem_raw + 3 * S::coef + S::red);

  const int tid = threadIdx.x, nthr = LY::WARPS * 32;
  const int lane = tid & 31, lg = lane % PG, warp = tid >> 5;
  const int cb = GW == 1 ? warp * LY::CPW + lane / PG : warp / GW;  // cell of this lane within the CTA
  const int gw = GW == 1 ? 0 : warp % GW;                            // which warp of the cell
  const int pidx = gw * 32 + lg;                                      // Gauss point of this lane
  const int i0 = blockIdx.x * CB, j = blockIdx.y, k = blockIdx.z;
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  const long long nc = m.ncell;
  const size_t row = ((size_t)k * ny + j) * nx;

  for (int e = tid; e < NC * CB; e += nthr) {
    const int cc = e % CB, comp = e / CB, i = i0 + cc;
    double q = 0, mR = 0, mT = 0;
    if (i < nx) {
      const size_t idx = (size_t)comp * nc + row + i;
      const double iM = inv_mass(comp % NM, cell_vol64(m, i, j, k));
      const double a = io.lamA[idx], b = io.lamB ? io.lamB[idx] : 0.0;
      q = Q[idx];
      mR = iM * (io.cLA * a + io.cLB * b);
      mT = iM * (io.cTA * a + io.cTB * b);
    }
    cq[comp][cc] = q;
    if (!FTO) cmuR[comp][cc] = mR;
    cmuT[comp][cc] = mT;
  }
  __syncthreads();

  const bool active = (pidx < NP) && (i0 + cb < nx);
  const int pp = active ? pidx : 0;
  const int pa[3] = {pp / (NQ * NQ), (pp / NQ) % NQ, pp % NQ};
  double L1[3][ORDER + 1], dL1[3][ORDER + 1];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double x = gauss_x(NQ, pa[d]);
#pragma unroll
    for (int n = 0; n <= ORDER; ++n) {
      L1[d][n] = leg<double>(n, x);
      dL1[d][n] = dleg<double>(n, x);
    }
  }
  const int icell = (i0 + cb < nx) ? i0 + cb : nx - 1;
  const double sc[3] = {cell_sc<double>(m, 0, icell), cell_sc<double>(m, 1, j), cell_sc<double>(m, 2, k)};
  const double w =
      active ? gauss_w(NQ, pa[0]) * gauss_w(NQ, pa[1]) * gauss_w(NQ, pa[2]) * cell_vol64(m, icell, j, k) : 0.0;

  // traces and flux cotangents: lambda_F_d[v] = w (2/h_d) sum_n dB_n/dr_d mu_R[v][n]
  double q[5], dq[3][5], lF[3][5], lT[3][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double s0 = 0, g[3] = {0, 0, 0}, f3[3] = {0, 0, 0}, t3[3] = {0, 0, 0};
#pragma unroll
    for (int mm = 0; mm < NM; ++mm) {
      const int e0 = mode_exp(mm, 0), e1 = mode_exp(mm, 1), e2 = mode_exp(mm, 2);
      const double c = cq[v * NM + mm][cb];
      const double dB[3] = {dL1[0][e0] * L1[1][e1] * L1[2][e2], L1[0][e0] * dL1[1][e1] * L1[2][e2],
                            L1[0][e0] * L1[1][e1] * dL1[2][e2]};
      s0 += c * (L1[0][e0] * L1[1][e1] * L1[2][e2]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        g[d] += c * dB[d];
        if (!FTO) f3[d] += dB[d] * cmuR[v * NM + mm][cb];
        t3[d] += dB[d] * cmuT[v * NM + mm][cb];
      }
    }
    q[v] = s0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dq[d][v] = g[d] * sc[d];
      lF[d][v] = w * sc[d] * f3[d];
      lT[d][v] = w * sc[d] * t3[d];
    }
  }

  // reverse mode of the interior flux (gks_point_adj.cuh): one backward sweep
  double gq[5], gdq[3][5], gmu = 0.0;
  interior_flux_vjp<double, FTO>(q, dq, gp, lF, lT, gq, gdq, gmu);
  if (!active) {
    gmu = 0.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      gq[v] = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) gdq[d][v] = 0.0;
    }
  }
  mured[tid] = gmu;

  // trace transpose summed over the cell's points (group butterfly), PG
  // outputs at a time: lane lg ends with output c0 + lg of each chunk
#pragma unroll
  for (int c0 = 0; c0 < NOP2; c0 += PG) {
    double val[PG];
#pragma unroll
    for (int oo = 0; oo < PG; ++oo) {
      const int o = c0 + oo;
      double c = 0.0;
      if (o < NC) {
        const int v = o / NM, mm = o % NM;
        const int e0 = mode_exp(mm, 0), e1 = mode_exp(mm, 1), e2 = mode_exp(mm, 2);
        c = (L1[0][e0] * L1[1][e1] * L1[2][e2]) * gq[v] + sc[0] * (dL1[0][e0] * L1[1][e1] * L1[2][e2]) * gdq[0][v] +
            sc[1] * (L1[0][e0] * dL1[1][e1] * L1[2][e2]) * gdq[1][v] +
            sc[2] * (L1[0][e0] * L1[1][e1] * dL1[2][e2]) * gdq[2][v];
      }
      val[oo] = c;
    }
    double outv[1];
    group_reduce<PG, PG>(val, outv, lg);
    red[cb][gw][c0 + lg] = outv[0];
  }
  __syncthreads();

  // add the faces' cotangents and the pass-through terms
  for (int o = tid; o < CB * NC; o += nthr) {
    const int cc = o % CB, comp = o / CB, i = i0 + cc;
    if (i >= nx) continue;
    const size_t cell = row + i, idx = (size_t)comp * nc + cell;
    double s = red[cc][0][comp];
#pragma unroll
    for (int g = 1; g < GW; ++g) s += red[cc][g][comp];
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      size_t up;
      if (D == 0)
        up = row + wrapm(i + 1, nx);
      else if (D == 1)
        up = ((size_t)k * ny + wrapm(j + 1, ny)) * nx + i;
      else
        up = ((size_t)wrapm(k + 1, nz) * ny + j) * nx + i;
      s += io.H[(((size_t)D * 2 + 1) * NC + comp) * nc + cell];  // this cell is right of its low face
      s += io.H[(((size_t)D * 2 + 0) * NC + comp) * nc + up];    // and left of its high face
    }
    if (io.addA) s += io.addA[idx];
    if (io.addB) s += io.addB[idx];
    io.out[idx] = s;
  }
  if (tid == 0) {
    double sm = 0.0;
    for (int t = 0; t < nthr; ++t) sm += mured[t];
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    io.mu_part[mu_offset + blk] = sm;
  }
}

// ---------------------------------------------------------------------------
// Gradient of E_k = 1/(rho0 |Omega|) sum w |K| |m|^2/(2 rho) (n_q^3 points):
// dE/dQ[v][n] = 1/(rho0 |Omega|) sum_p w |K| B_n(p) de/dq_v, with
// de/drho = -|m|^2/(2 rho^2), de/dm_d = m_d / rho, de/drhoE = 0.
// ---------------------------------------------------------------------------
template <int ORDER, int NQ>
__global__ void __launch_bounds__(RED_THREADS) k_ek_vjp(const double* __restrict__ Q, const MeshDev m, double scale,
                                                        double* __restrict__ out) {
  constexpr int NM = n_modes(ORDER);
  const long long nc = m.ncell;
  for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < nc; c += (long long)gridDim.x * RED_THREADS) {
    const double cw = cell_weight(m, c) * scale;  // |K| / (rho0 |Omega|) (|K| in scale on a uniform mesh)
    double co[4][NM], g[5][NM];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) co[v][mm] = Q[(size_t)(v * NM + mm) * nc + c];
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) g[v][mm] = 0.0;
#pragma unroll
    for (int a = 0; a < NQ; ++a)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int cz = 0; cz < NQ; ++cz) {
          double qv[4] = {0, 0, 0, 0}, B[NM];
#pragma unroll
          for (int mm = 0; mm < NM; ++mm) {
            B[mm] = leg<double>(mode_exp(mm, 0), gauss_x(NQ, a)) * leg<double>(mode_exp(mm, 1), gauss_x(NQ, b)) *
                    leg<double>(mode_exp(mm, 2), gauss_x(NQ, cz));
#pragma unroll
            for (int v = 0; v < 4; ++v) qv[v] += co[v][mm] * B[mm];
          }
          const double wq = gauss_w(NQ, a) * gauss_w(NQ, b) * gauss_w(NQ, cz) * cw;
          const double ir = 1.0 / qv[0];
          const double m2 = qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3];
          const double de[4] = {-0.5 * m2 * ir * ir, qv[1] * ir, qv[2] * ir, qv[3] * ir};
#pragma unroll
          for (int mm = 0; mm < NM; ++mm)
#pragma unroll
            for (int v = 0; v < 4; ++v) g[v][mm] += wq * B[mm] * de[v];
        }
#pragma unroll
    for (int v = 0; v < 5; ++v)
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) out[(size_t)(v * NM + mm) * nc + c] = g[v][mm];
  }
}

// sum of the viscosity-cotangent partials (fixed order), added to *acc
__global__ void k_mu_sum(const double* __restrict__ part, long long n, double* __restrict__ acc) {
  __shared__ double sh[RED_THREADS];
  double s = 0.0;
  for (long long b = threadIdx.x; b < n; b += RED_THREADS) s += part[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = RED_THREADS / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += sh[0];
}

}  // namespace dghgks
