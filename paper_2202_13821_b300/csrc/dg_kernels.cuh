// DG-HGKS residual kernels (Sec. 3 of arXiv:2202.13821, Eqs. operator,
// surface, volume, two-stage), templated on the flux arithmetic R (double,
// or float in the FP32-mixed path), the degree ORDER and the Gauss count NQ.
//
// One stage = 3 face launches (one per normal direction) + 1 cell launch:
//
//   k_face<D>: a CTA owns FB consecutive faces along x normal to axis D.  While
//     staging the two cells of each face (coalesced loads), it contracts
//     their modal coefficients along the normal, so each side's trace is a
//     2-D polynomial in the tangential coordinates (value and normal
//     derivative).  Lanes run over faces; in FP32 a thread takes the n_q
//     Gauss points of one row of its face in turn (n_q warps per CTA), in
//     FP64 one warp per Gauss point.  At each of its points a thread
//     evaluates Q_h and grad Q_h on both sides, computes F_b and d_t F_b there
//     (Eq. flux, local frame with the normal first), and the CTA projects
//     w |Gamma| F onto the NT tangential Legendre products of the face in
//     shared memory.  Only those face moments G reach HBM (10 x NT values per
//     face); point values never do.
//
//   k_cell<MODE>: a group of lanes owns one cell, one lane per Gauss point
//     (a warp per cell at n_q = 3, four cells per warp at n_q = 2, two warps
//     per cell at n_q = 4).  Each lane evaluates Q_h and grad Q_h at its point
//     (cell-major coefficient rows and, at k <= 2, a per-CTA table of the
//     basis at the points, both read with 16-byte loads) and the interior
//     flux of Eq. (flux-2) there; the volume projection w |K| F . grad B_n is
//     summed over the cell's lanes in a fixed order (one cell per warp:
//     transposed through shared memory, each lane summing one output column;
//     otherwise by recursive-halving warp butterflies; no atomics).  The
//     cell's lanes then add the six faces' moments with
//     the sign and parity of Eq. (operator) (the cell is right of its low
//     face: +(-1)^{n_D} G, left of its high face: -G), multiplies by the
//     diagonal inverse mass matrix, and applies the epilogue:
//       MODE 0: write L = M^-1 R and L_t = M^-1 R_t
//       MODE 1: Q* = Q^n + dt/2 L + dt^2/8 L_t, inc = dt L + dt^2/6 L_t
//       MODE 2: Q^{n+1} = Q^n + inc + dt^2/3 L_t(Q*)
//     The epilogue runs in the precision E: E = R (FP64, and the FP32-mixed
//     path) stores Q* and inc in the flux precision, and the accumulation into
//     the stored FP64 state is the one FP64 operation (on B300 an FP64
//     instruction costs ~64 FP32 ones).  E = double with R = float (the
//     FP32-flux / FP64-stage path): the volume sums and their assembly with
//     the face moments are FP32 (the mode-0 outputs' face terms summed
//     exactly, for FP64-level conservation), M^-1, Q* and inc are FP64 (Q*
//     formed from the FP64 state and stored rounded to R, its precision as an
//     input of the stage-2 flux kernels; inc stored in FP64).
//
// Each face is computed exactly once and written by exactly one CTA, and
// every residual coefficient is summed in a fixed order: results are
// bit-reproducible from run to run (no floating-point atomics).
// A non-physical state (rho <= 0 or p <= 0) sets bit 0 of *flag; a wait of
// the persistent cell kernel on one of its shared-memory barriers that has
// not completed within 2 s (it never should) sets bit 1 and ends the kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dg_tables.cuh"
#include "gks_point.cuh"

namespace dghgks {

struct MeshDev {
  int nx, ny, nz;
  long long ncell;
  double h[3];
  double vol;
  // the same in single precision, precomputed on the host for the FP32 path
  float sc_f[3];    // 2 / h_d
  float area_f[3];  // |Gamma| of a face normal to d
  float vol_f;
  double ivol;      // 1 / |K|
  float ivol_f;
  // Rectilinear (non-uniform) meshes: per axis d, the n_d cell widths followed
  // by the n_d values 2 / width, in FP64 and FP32.  All null on a uniform mesh,
  // where the scalars above hold.
  const double* geo64[3];
  const float* geo32[3];
};

__device__ __forceinline__ bool mesh_nonuniform(const MeshDev& m) { return m.geo64[0] != nullptr; }
__device__ __forceinline__ int mesh_n(const MeshDev& m, int d) { return d == 0 ? m.nx : (d == 1 ? m.ny : m.nz); }

// per-precision access to the mesh scales
template <class R>
__device__ __forceinline__ R mesh_sc(const MeshDev& m, int d) {
  return R(2) / (R)m.h[d];
}
template <>
__device__ __forceinline__ float mesh_sc<float>(const MeshDev& m, int d) {
  return m.sc_f[d];
}
template <class R>
__device__ __forceinline__ R mesh_area(const MeshDev& m, int d) {
  return (R)(m.vol / m.h[d]);
}
template <>
__device__ __forceinline__ float mesh_area<float>(const MeshDev& m, int d) {
  return m.area_f[d];
}
template <class R>
__device__ __forceinline__ R mesh_vol(const MeshDev& m) {
  return (R)m.vol;
}
template <>
__device__ __forceinline__ float mesh_vol<float>(const MeshDev& m) {
  return m.vol_f;
}
template <class R>
__device__ __forceinline__ R mesh_ivol(const MeshDev& m) {
  return (R)m.ivol;
}
template <>
__device__ __forceinline__ float mesh_ivol<float>(const MeshDev& m) {
  return m.ivol_f;
}
template <class R>
__device__ __forceinline__ const R* mesh_geo(const MeshDev& m, int d) {
  return reinterpret_cast<const R*>(m.geo64[d]);
}
template <>
__device__ __forceinline__ const float* mesh_geo<float>(const MeshDev& m, int d) {
  return m.geo32[d];
}
// width of cell c along axis d
template <class R>
__device__ __forceinline__ R cell_w(const MeshDev& m, int d, int c) {
  return mesh_nonuniform(m) ? __ldg(mesh_geo<R>(m, d) + c) : (R)m.h[d];
}
// 2 / width of cell c along axis d (the reference-to-physical gradient scale)
template <class R>
__device__ __forceinline__ R cell_sc(const MeshDev& m, int d, int c) {
  return mesh_nonuniform(m) ? __ldg(mesh_geo<R>(m, d) + mesh_n(m, d) + c) : mesh_sc<R>(m, d);
}
// |Gamma| of the face normal to d whose tangential cells are c1 (axis tan1) and c2 (axis tan2)
template <class R>
__device__ __forceinline__ R face_area(const MeshDev& m, int d, int c1, int c2) {
  return mesh_nonuniform(m) ? cell_w<R>(m, tan1(d), c1) * cell_w<R>(m, tan2(d), c2) : mesh_area<R>(m, d);
}
// FP64 volume of cell (i, j, k)
__device__ __forceinline__ double cell_vol64(const MeshDev& m, int i, int j, int k) {
  return mesh_nonuniform(m) ? __ldg(m.geo64[0] + i) * __ldg(m.geo64[1] + j) * __ldg(m.geo64[2] + k) : m.vol;
}
// FP64 volume of cell c (linear index) on a rectilinear mesh; 1 on a uniform
// mesh, where the reductions scale by the common volume at the end
__device__ __forceinline__ double cell_weight(const MeshDev& m, long long c) {
  if (!mesh_nonuniform(m)) return 1.0;
  const int i = (int)(c % m.nx), j = (int)((c / m.nx) % m.ny), k = (int)(c / ((long long)m.nx * m.ny));
  return __ldg(m.geo64[0] + i) * __ldg(m.geo64[1] + j) * __ldg(m.geo64[2] + k);
}

constexpr int FB = 32;  // faces per CTA in k_face

// Register cap of k_face.  The register file of an SM is split between its
// four sub-partitions (16384 registers each) and a CTA's warps are spread
// over them, so the cap for C resident CTAs of W warps is
// 16384 / (ceil(C W / 4) x 32), rounded down to a multiple of 8.
// FP32: a thread takes the NQ Gauss points of one row of its face in turn
// (NQ warps per CTA), and the CTAs per SM are chosen so that 128 registers
// hold the kernel without spills: 8 CTAs at n_q = 2, 5 at n_q = 3, 4 at
// n_q = 4.  At 256^3, n_q = 3, a face launch took 3-6% longer with 4 CTAs
// at 156 registers, 22% longer with 8 CTAs at 80 registers (spills) and 24%
// longer with one warp per Gauss point (9 warps, 72 registers, spills).
// FP64 (bound by the FP64 pipe): one warp per Gauss point, 1 CTA.
#ifndef FACE_CTAS_NQ3
#define FACE_CTAS_NQ3 5
#endif
template <class R, int NQ>
constexpr int face_ppt() {
  return (sizeof(R) == 4 && NQ >= 2) ? NQ : 1;
}
template <class R, int NQ>
constexpr int face_max_regs() {
  constexpr int warps = (FB * NQ * NQ / face_ppt<R, NQ>() + 31) / 32;
  constexpr int ctas = sizeof(R) == 4 ? (NQ == 2 ? 8 : NQ == 3 ? FACE_CTAS_NQ3 : 4) : 1;
  constexpr int per_part = (warps * ctas + 3) / 4;
  constexpr int cap = 16384 / (per_part * 32) / 8 * 8;
  return cap > 255 ? 255 : cap;
}

// Per side and variable, a face stages the traces of its cell as two
// polynomials in the tangential coordinates: the value at r_D = +-1 (NT
// tangential modes) and the normal derivative there (degree ORDER - 1, NN
// modes), each coefficient a signed sum of the cell's modes along D.
// A face's polynomials are contiguous in its row, each variable's NK values
// padded to whole 16-byte groups (VP values), the row pitch an odd number of
// 16-byte groups, so that the points read them with conflict-free 16-byte loads.
template <class R, int ORDER, int NQ>
struct FaceSmem {
  static constexpr int NM = n_modes(ORDER), NT = n_tmodes(ORDER), NN = n_tmodes(ORDER - 1), NK = NT + NN;
  static constexpr int NP = NQ * NQ, W16 = 16 / sizeof(R);
  static constexpr int PPT = face_ppt<R, NQ>(), THREADS = FB * NP / PPT;  // points per thread, CTA size
  static constexpr int VP = (NK + W16 - 1) / W16 * W16;
  static constexpr int PITCH = ((5 * VP / W16) % 2 == 1) ? 5 * VP : 5 * VP + W16;
  static constexpr size_t coef = sizeof(R) * PITCH * FB;  // one side
  static constexpr size_t fs = sizeof(R) * 10 * NP * FB;
  static constexpr size_t bytes = 2 * coef + fs;
  static_assert(sizeof(R) * FB * 10 * NT <= 2 * coef, "face moments must fit the staging area");
};

// N consecutive values (N a multiple of 16 / sizeof(R), 16-byte aligned) from shared memory
template <int N, class R>
__device__ __forceinline__ void lds16(const R* p, R (&c)[N]) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 q = reinterpret_cast<const float4*>(p)[i];
      c[4 * i] = q.x, c[4 * i + 1] = q.y, c[4 * i + 2] = q.z, c[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const double2 q = reinterpret_cast<const double2*>(p)[i];
      c[2 * i] = q.x, c[2 * i + 1] = q.y;
    }
  }
}

__device__ __forceinline__ int wrapm(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---------------------------------------------------------------------------
// Face kernel
// ---------------------------------------------------------------------------
// FTO (the stage-2 pass of S2O4, which needs L_t(Q*) only): the F_t moments
// alone are projected and stored; F is left to dead-code elimination.
template <class R, int ORDER, int NQ, int D, class Tin, bool FTO = false>
__global__ void __launch_bounds__(FaceSmem<R, ORDER, NQ>::THREADS) __maxnreg__((face_max_regs<R, NQ>()))
    k_face(const Tin* __restrict__ Q, R* __restrict__ G, const GasPar<R> gp, const MeshDev m,
           unsigned* __restrict__ flag) {
  using S = FaceSmem<R, ORDER, NQ>;
  constexpr int NM = S::NM, NT = S::NT, NN = S::NN, NP = S::NP, VP = S::VP, PITCH = S::PITCH;
  constexpr int PPT = S::PPT, NTHR = S::THREADS, NPW = NP / PPT;  // NPW threads per face
  constexpr int T1 = tan1(D), T2 = tan2(D);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R(*cL)[PITCH] = reinterpret_cast<R(*)[PITCH]>(smem_raw);  // [face][var VP + poly value]
  R(*cR)[PITCH] = reinterpret_cast<R(*)[PITCH]>(smem_raw + S::coef);
  R(*Fs)[NP][FB] = reinterpret_cast<R(*)[NP][FB]>(smem_raw + 2 * S::coef);

  const int tid = threadIdx.x;
  const int f = tid % FB, pw = tid / FB;
  const int i0 = blockIdx.x * FB, j = blockIdx.y, k = blockIdx.z;
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  const long long nc = m.ncell;

  // stage the face polynomials of the left (-e_D; traces at r_D = +1) and
  // right (r_D = -1) cells of each face: P_n(+1) = 1, P_n(-1) = (-1)^n,
  // P'_n(+1) = n(n+1)/2, P'_n(-1) = (-1)^(n+1) n(n+1)/2
  for (int e = tid; e < 2 * 5 * FB; e += NTHR) {
    const int ff = e % FB, rest = e / FB, v = rest % 5, side = rest / 5;
    const int i = i0 + ff;
    R Vt[NT], Nt[NN];
#pragma unroll
    for (int t = 0; t < NT; ++t) Vt[t] = R(0);
#pragma unroll
    for (int t = 0; t < NN; ++t) Nt[t] = R(0);
    if (i < nx) {
      int ci = i, cj = j, ck = k;
      if (side == 0) {
        if (D == 0) ci = wrapm(i - 1, nx);
        if (D == 1) cj = wrapm(j - 1, ny);
        if (D == 2) ck = wrapm(k - 1, nz);
      }
      const Tin* src = Q + (size_t)(v * NM) * nc + ((size_t)ck * ny + cj) * nx + ci;
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) {
        const R c = (R)__ldg(src + (size_t)mm * nc);
        const int nD = mode_exp(mm, D), t = tmode_index(mode_exp(mm, T1), mode_exp(mm, T2));
        const bool neg = side == 1 && (nD % 2 == 1);
        Vt[t] += neg ? -c : c;
        if (nD > 0) {
          const R dc = R(nD * (nD + 1) / 2) * c;
          Nt[t] += (side == 1 && nD % 2 == 0) ? -dc : dc;
        }
      }
    }
    // (16-byte stores: the variable's VP values are 16-byte aligned)
    R vals[VP];
#pragma unroll
    for (int t = 0; t < VP; ++t) vals[t] = t < NT ? Vt[t] : (t < NT + NN ? Nt[t - NT] : R(0));
    R* dst = (side == 0 ? cL : cR)[ff] + v * VP;
#pragma unroll
    for (int q = 0; q < VP * (int)sizeof(R) / 16; ++q) {
      if constexpr (sizeof(R) == 4)
        reinterpret_cast<float4*>(dst)[q] = make_float4(vals[4 * q], vals[4 * q + 1], vals[4 * q + 2], vals[4 * q + 3]);
      else
        reinterpret_cast<double2*>(dst)[q] = make_double2(vals[2 * q], vals[2 * q + 1]);
    }
  }
  __syncthreads();

  const int i = i0 + f;
  const bool active = i < nx;
  // gradient scales: along D those of the left and right cells, tangential
  // ones shared by both cells (rectilinear mesh)
  const int ic = active ? i : 0;
  const int cidx[3] = {ic, j, k};
  const int nAx = D == 0 ? nx : (D == 1 ? ny : nz);
  const R sDs[2] = {cell_sc<R>(m, D, wrapm(cidx[D] - 1, nAx)), cell_sc<R>(m, D, cidx[D])};
  const R s1 = cell_sc<R>(m, T1, cidx[T1]), s2 = cell_sc<R>(m, T2, cidx[T2]);
  const R area = face_area<R>(m, D, cidx[T1], cidx[T2]);
#pragma unroll 1
  for (int pp = 0; pp < PPT; ++pp) {
  const int p = pw * PPT + pp;  // this thread's Gauss point of the face
  const int a = p / NQ, b = p % NQ;
  const R xa = gauss_xr<R>(NQ, a), xb = gauss_xr<R>(NQ, b);
  // tangential basis at this point: phi_t, d phi_t / d r_1, d phi_t / d r_2
  R Bt[NT], B1[NT], B2[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int tp = tmode_p(t), tq = tmode_q(t);
    Bt[t] = leg<R>(tp, xa) * leg<R>(tq, xb);
    B1[t] = tp > 0 ? dleg<R>(tp, xa) * leg<R>(tq, xb) : R(0);
    B2[t] = tq > 0 ? leg<R>(tp, xa) * dleg<R>(tq, xb) : R(0);
  }

  // Each side in turn: traces of the left cell (side 0) or the right cell
  // (side 1) from its face polynomials, rotated to the local frame (axes D,
  // D+1, D+2 cyclic, momentum alike), folded into the side sums of Eq. (flux).
  constexpr int A0 = D, A1 = (D + 1) % 3, A2 = (D + 2) % 3;
  const bool pr_fix = (gp.pr_fix != R(0));
  SideSums<R> sums;
  iface_zero(sums);
  bool ok = true;
#pragma unroll 1  // sides in turn, not interleaved: fewer live registers
  for (int side = 0; side < 2; ++side) {
    const R* cs = (side == 0 ? cL : cR)[f];
    R q[5], dq[3][5];  // global axes
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      R cv[VP];
      lds16(cs + v * VP, cv);
      R s0 = R(0), gD = R(0), g1 = R(0), g2 = R(0);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const R c = cv[t];
        s0 += c * Bt[t];
        if (tmode_p(t) > 0) g1 += c * B1[t];
        if (tmode_q(t) > 0) g2 += c * B2[t];
        if (t < NN) gD += cv[NT + t] * Bt[t];
      }
      q[v] = s0;
      dq[D][v] = gD * sDs[side];
      dq[T1][v] = g1 * s1;
      dq[T2][v] = g2 * s2;
    }
    R ql[5], dql[3][5];
    const int ax[3] = {A0, A1, A2};
    ql[0] = q[0];
    ql[1] = q[1 + A0];
    ql[2] = q[1 + A1];
    ql[3] = q[1 + A2];
    ql[4] = q[4];
#pragma unroll
    for (int ii = 0; ii < 3; ++ii) {
      const R* src = dq[ax[ii]];
      dql[ii][0] = src[0];
      dql[ii][1] = src[1 + A0];
      dql[ii][2] = src[1 + A1];
      dql[ii][3] = src[1 + A2];
      dql[ii][4] = src[4];
    }
    ok = iface_side<R>(side == 0 ? 1 : -1, ql, dql, gp, pr_fix, sums) && ok;
  }
  R Fl[5], Ftl[5];
  ok = iface_finish(sums, gp, Fl, Ftl) && ok;
  if (active && !ok) atomicOr(flag, 1u);
  const R w = active ? gauss_wr<R>(NQ, a) * gauss_wr<R>(NQ, b) * area : R(0);
  if (!FTO) {
    Fs[0][p][f] = w * Fl[0];
    Fs[1 + A0][p][f] = w * Fl[1];
    Fs[1 + A1][p][f] = w * Fl[2];
    Fs[1 + A2][p][f] = w * Fl[3];
    Fs[4][p][f] = w * Fl[4];
  }
  Fs[5][p][f] = w * Ftl[0];
  Fs[6 + A0][p][f] = w * Ftl[1];
  Fs[6 + A1][p][f] = w * Ftl[2];
  Fs[6 + A2][p][f] = w * Ftl[3];
  Fs[9][p][f] = w * Ftl[4];
  }
  __syncthreads();

  // tangential projection G[D][face][c][t] = sum_p Fs[c][p] phi_t(p): the
  // thread with point index p takes components c = p, p + NP, ...; the
  // Legendre products phi_t(p) are compile-time constants.  The CTA's faces
  // are consecutive in G (face-major layout), so the moments are gathered in
  // shared memory (over the coefficient staging area, free after the
  // barrier above) and written as one contiguous block.
  R(*Gs)[10][NT] = reinterpret_cast<R(*)[10][NT]>(smem_raw);
  for (int c = (FTO ? 5 : 0) + pw; c < 10; c += NPW) {
    R fv[NP];
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) fv[pp] = Fs[c][pp][f];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      R s = R(0);
#pragma unroll
      for (int pp = 0; pp < NP; ++pp)
        s += fv[pp] * (leg<R>(tmode_p(t), gauss_xr<R>(NQ, pp / NQ)) * leg<R>(tmode_q(t), gauss_xr<R>(NQ, pp % NQ)));
      Gs[f][c][t] = s;
    }
  }
  __syncthreads();
  // (in the widest vector units, up to 16 bytes, that the block or its F_t
  // half and the face offsets are multiples of)
  const int nf = nx - i0 < FB ? nx - i0 : FB;
  R* const dst = G + ((size_t)D * nc + ((size_t)k * ny + j) * nx + i0) * (10 * NT);
  const R* const src = &Gs[0][0][0];
  constexpr int BYTES = (FTO ? 5 : 10) * NT * (int)sizeof(R);  // bytes written per face
  constexpr int UB = BYTES % 16 == 0 ? 16 : (BYTES % 8 == 0 ? 8 : 4);
  using V = typename std::conditional<UB == 16, uint4, typename std::conditional<UB == 8, uint2, unsigned>::type>::type;
  constexpr int PV = BYTES / UB, FS = 10 * NT * (int)sizeof(R) / UB;  // vectors per face, face stride
  V* const dv = reinterpret_cast<V*>(dst);
  const V* const sv = reinterpret_cast<const V*>(src);
  if (FTO) {
    for (int e = tid; e < nf * PV; e += NTHR) {
      const int ff = e / PV, r = e % PV;
      dv[ff * FS + PV + r] = sv[ff * FS + PV + r];
    }
  } else {
    for (int e = tid; e < nf * PV; e += NTHR) dv[e] = sv[e];
  }
}

// ---------------------------------------------------------------------------
// Cell kernel
// ---------------------------------------------------------------------------
enum { MODE_RESIDUAL = 0, MODE_STAGE1 = 1, MODE_STAGE2 = 2 };

// Thread layout of k_cell: the NQ^3 Gauss points of a cell are spread over
// GW warps (GW = 1 for NQ <= 3, 2 for NQ = 4), one lane per point; at
// NQ <= 3 a group of PG lanes holds one cell (PG = 8 at NQ = 2: four cells
// per warp).  Spare lanes carry zeros.  8 warps per CTA.
template <int ORDER, int NQ>
struct CellLayout {
  static constexpr int NP = NQ * NQ * NQ;
  static constexpr int GW = (NP + 31) / 32;          // warps per cell
  static constexpr int PG = NP <= 8 ? 8 : 32;        // lanes of a reduction group
  static constexpr int CPW = GW == 1 ? 32 / PG : 1;  // cells per warp
  static constexpr int WARPS = 8;
  static constexpr int CB = GW == 1 ? CPW * WARPS : WARPS / GW;  // cells per CTA
  static constexpr int NM = n_modes(ORDER);
  static constexpr int NOUT = 5 * (NM - 1);                 // volume outputs (mode 0 has no gradient)
  static constexpr int NOP = (NOUT + PG - 1) / PG * PG;      // padded to the group width
  static_assert(NP <= 64, "k_cell handles up to 4^3 points per cell");
};

// Basis of k_cell at a Gauss point p: the values phi_n(p), the gradients
// d phi_n / d r_d (p) and the weight product w_a w_b w_c, as products of the
// Legendre values at the Gauss nodes in the flux precision.  The persistent
// one-warp-per-cell layout at k <= 2 keeps them in shared memory, one row per
// point (built once per CTA; a lane loads its row with 16-byte loads):
//   [0, POFF): the gradients of the pairs (n, d) with a non-zero exponent
//     along d, at slot d NGD + (index of the mode with that exponent lowered
//     by one; NGD = modes of degree k - 1),
//   [POFF, WOFF): phi_n,  WOFF: the weight,
// each section padded to a multiple of 4 values.  Otherwise (k = 3, whose
// row would crowd the registers, or a cell over two warps) a lane forms them
// from the Legendre values held in registers.
template <class R, int ORDER, int NQ>
struct CellBasis {
  static constexpr int NM = n_modes(ORDER), NGD = n_modes(ORDER - 1);
  static constexpr int POFF = (3 * NGD + 3) / 4 * 4, WOFF = POFF + (NM + 3) / 4 * 4, BW = WOFF + 4;
  static constexpr int gslot(int n, int d) {
    return d * NGD + mode_index2(mode_exp(n, 0) - (d == 0), mode_exp(n, 1) - (d == 1), mode_exp(n, 2) - (d == 2));
  }
  R L[3][ORDER + 1], dL[3][ORDER + 1], w;
  __device__ __forceinline__ explicit CellBasis(int p) {
    const int pa[3] = {p / (NQ * NQ), (p / NQ) % NQ, p % NQ};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R x = gauss_xr<R>(NQ, pa[d]);
#pragma unroll
      for (int n = 0; n <= ORDER; ++n) {
        L[d][n] = leg<R>(n, x);
        dL[d][n] = dleg<R>(n, x);
      }
    }
    w = gauss_wr<R>(NQ, pa[0]) * gauss_wr<R>(NQ, pa[1]) * gauss_wr<R>(NQ, pa[2]);
  }
  // (mm, d compile-time after unrolling)
  __device__ __forceinline__ R phi(int mm) const {
    return L[0][mode_exp(mm, 0)] * L[1][mode_exp(mm, 1)] * L[2][mode_exp(mm, 2)];
  }
  __device__ __forceinline__ R grad(int mm, int d) const {
    return (d == 0 ? dL[0][mode_exp(mm, 0)] : L[0][mode_exp(mm, 0)]) *
           (d == 1 ? dL[1][mode_exp(mm, 1)] : L[1][mode_exp(mm, 1)]) *
           (d == 2 ? dL[2][mode_exp(mm, 2)] : L[2][mode_exp(mm, 2)]);
  }
};

template <class R, int ORDER, int NQ, class Tin = R, class E = R, int MODE = MODE_RESIDUAL>
struct CellSmem {
  using LY = CellLayout<ORDER, NQ>;
  static constexpr int NM = LY::NM, NC = 5 * NM, CB = LY::CB;
  // the coefficients of a tile are staged cell-major: per cell a row of the
  // 5 variables' NM modes, each variable padded to NMP values (v NMP + n), so
  // that a lane reads a variable's modes with 16-byte loads
  static constexpr int NMP = (NM + 3) / 4 * 4, NCP = 5 * NMP;
  // GW = 1: NBUF staging buffers of the input type (cp.async targets), plus a
  // converted copy when the input is not in the flux precision; GW > 1: one
  // buffer in the flux precision.
  // (three when DECOUPLED: a warp may run one tile ahead of the slowest warp
  // of its CTA; two when a CTA barrier per tile orders the passes)
#ifndef CELL_DECOUPLE_STAGE2
#define CELL_DECOUPLE_STAGE2 0
#endif
  static constexpr bool DECOUPLED = MODE != MODE_STAGE2 || CELL_DECOUPLE_STAGE2;
  static constexpr int NBUF = DECOUPLED ? 3 : 2;
  // output buffers: DECOUPLED, four (the buffer a tile writes was written out
  // by every thread before it finished the tile two back)
  static constexpr int NOBUF = DECOUPLED ? 4 : 2;
  static constexpr size_t raw = LY::GW == 1 ? NBUF * sizeof(Tin) * NCP * CB : 0;
  static constexpr size_t cvt = (LY::GW == 1 && std::is_same<Tin, R>::value) ? 0 : sizeof(R) * NCP * CB;
  // cross-warp partial sums (only when a cell spans two warps)
  static constexpr size_t red = LY::GW == 1 ? 0 : sizeof(R) * CB * LY::GW * 2 * LY::NOP;
  // GW = 1: the outputs of a tile (NKO kinds: two, one at stage 2; NC x CB),
  // in NOBUF buffers, so that they leave as rows of CB consecutive cells
  static constexpr int NKO = MODE == MODE_STAGE2 ? 1 : 2;
  static constexpr size_t out = LY::GW == 1 ? sizeof(E) * NOBUF * NKO * NC * CB : 0;
  // one cell per warp (n_q = 3): the volume projection is transposed through
  // shared memory, a row per Gauss point and warp holding the point's
  // contributions to 32 outputs, (F, F_t) pairs (F_t alone at stage 2); the
  // row stride is padded by 16 bytes (conflict-free 16-byte stores along a
  // row and 8-byte loads down a column)
  static constexpr bool TRANS = LY::GW == 1 && LY::PG == 32;
  static constexpr int TS = (MODE == MODE_STAGE2 ? 32 : 64) + 16 / (int)sizeof(R);
  static constexpr size_t tr = TRANS ? sizeof(R) * LY::WARPS * LY::NP * TS : 0;
  // per output (v, n): its offsets v NT + t_D(n) in the face blocks normal to
  // D = 0, 1, 2 and the parity signs (-1)^{n_D}; M^-1 per mode; per mode the
  // tangential indices and signs again as ints (cells spanning two warps)
  static constexpr size_t tabs = 16 * NC + sizeof(R) * 4 * NC + sizeof(E) * NM + sizeof(int) * 6 * NM;
  // the basis table (CellBasis), one row per Gauss point (persistent layout, k <= 2)
  static constexpr bool TABLE = LY::GW == 1 && ORDER <= 2;
  static constexpr size_t bt = TABLE ? sizeof(R) * LY::NP * CellBasis<R, ORDER, NQ>::BW : 0;
  static constexpr size_t cvt_off = raw, red_off = raw + cvt, out_off = red_off + red, tr_off = out_off + out,
                          bt_off = tr_off + tr, tab_off = bt_off + bt;
  // GW = 1: the mbarriers of the persistent tile loop, NBUF each of full
  // (a tile's coefficients staged) and done (a tile finished by every warp)
  static constexpr size_t bar_off = (tab_off + tabs + 7) / 8 * 8;
  static constexpr size_t bytes = bar_off + (LY::GW == 1 && DECOUPLED ? 2 * NBUF * sizeof(unsigned long long) : 0);
  static_assert(cvt_off % 16 == 0 && red_off % 16 == 0 && out_off % 16 == 0, "16-byte aligned staging");
  static_assert(tr_off % 16 == 0 && tr % 16 == 0, "16-byte aligned transpose rows");
  static_assert(bt_off % 16 == 0 && tab_off % 16 == 0, "16-byte aligned basis rows and tables");
};

// Recursive-halving butterfly over the PG lanes of a group: in[N] per lane ->
// out[N/2] per lane after one exchange with the partner lane ^ M.  Lanes with
// the M bit set keep the upper half.
template <int N, int M, class R>
__device__ __forceinline__ void halve(const R (&in)[N], R (&out)[N / 2], bool upper) {
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    const R keep = upper ? in[j + N / 2] : in[j];
    const R send = upper ? in[j] : in[j + N / 2];
    out[j] = keep + __shfl_xor_sync(0xffffffffu, send, M);
  }
}

// Reduce the per-lane contributions val[NOP] over the PG lanes of the group:
// lane lg (0..PG-1) ends with the sums of outputs [RPL*lg, RPL*lg + RPL).
template <int NOP, int PG, class R>
__device__ __forceinline__ void group_reduce(const R (&val)[NOP], R (&out)[NOP / PG], int lg) {
  if constexpr (PG == 32) {
    R a[NOP / 2], b[NOP / 4], c[NOP / 8], d[NOP / 16];
    halve<NOP, 16>(val, a, lg & 16);
    halve<NOP / 2, 8>(a, b, lg & 8);
    halve<NOP / 4, 4>(b, c, lg & 4);
    halve<NOP / 8, 2>(c, d, lg & 2);
    halve<NOP / 16, 1>(d, out, lg & 1);
  } else {
    R a[NOP / 2], b[NOP / 4];
    halve<NOP, 4>(val, a, lg & 4);
    halve<NOP / 2, 2>(a, b, lg & 2);
    halve<NOP / 4, 1>(b, out, lg & 1);
  }
}

// cp.async (global -> shared, 4 or 8 bytes, bypassing registers); zfill:
// with valid = false nothing is read and the destination is zeroed.
template <class T>
__device__ __forceinline__ void cp_async_zfill(T* smem, const T* gmem, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? (int)sizeof(T) : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem), "n"(sizeof(T)), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared-memory mbarriers (CTA scope).  mbar_wait is bounded: it gives up
// after kMbarWaitNs of global time, or after kMbarMaxPolls polls whatever the
// timer says, and returns false.
constexpr unsigned long long kMbarWaitNs = 2000000000ull;
constexpr int kMbarMaxPolls = 1 << 24;
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b)) : "memory");
}
// arrives on b once every cp.async this thread has issued so far has completed
__device__ __forceinline__ void cp_async_mbar_arrive(unsigned long long* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  const unsigned a = smem_u32(b);
  unsigned long long t0 = 0;
  for (int it = 0;; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (it == 0)
      t0 = now;
    else if (now - t0 > kMbarWaitNs || it > kMbarMaxPolls)
      return false;
  }
}

// Accumulators of a cell output's face terms (sg * lo - hi per face, sg = +-1):
// PlainAcc sums in A; ExactAcc (FP32 terms) keeps the sum as an unevaluated
// pair s + e of FP32 numbers by error-free transformations (TwoSum, Knuth,
// TAOCP vol. 2, 4.2.2), so the FP64 value of s + e equals the exact sum to
// within about 1e-14 relative (the rounding of the small e only).
template <class A>
struct PlainAcc {
  A v;
  __device__ __forceinline__ explicit PlainAcc(A x) : v(x) {}
  template <class R>
  __device__ __forceinline__ void add(R sg, R lo, R hi) {
    v += (A)sg * (A)lo - (A)hi;
  }
  template <class E>
  __device__ __forceinline__ E get() const {
    return (E)v;
  }
};
struct ExactAcc {
  float s, e;
  __device__ __forceinline__ explicit ExactAcc(float x) : s(x), e(0.f) {}
  __device__ __forceinline__ void two_sum(float t) {
    const float a = s, x = __fadd_rn(a, t), bb = __fsub_rn(x, a);
    e = __fadd_rn(e, __fadd_rn(__fsub_rn(a, __fsub_rn(x, bb)), __fsub_rn(t, bb)));
    s = x;
  }
  __device__ __forceinline__ void add(float sg, float lo, float hi) {
    two_sum(sg * lo);  // exact: sg = +-1
    two_sum(-hi);
  }
  template <class E>
  __device__ __forceinline__ E get() const {
    return (E)s + (E)e;
  }
};

// Buffers of the cell-kernel epilogue (E: its precision, see the header).
//   MODE 0: L, Lt (FP64, caller's)
//   MODE 1: Qs = Q* in the flux precision R (the stage-2 kernels read Q* in R)
//           and inc = dt L + dt^2/6 L_t in E; with E = double, Q* is formed
//           from the FP64 state Qn
//   MODE 2: Qn (FP64 state, updated in place) += inc + dt^2/3 L_t(Q*); when Qf
//           is not null, also Qf = the updated state rounded to R (the next
//           step's stage-1 kernels read it instead of converting Qn)
template <class R, class E = R>
struct StageIO {
  double* L;
  double* Lt;
  R* Qs;
  E* inc;
  double* Qn;
  R* Qf;
};

// Resident CTAs of k_cell per SM requested from the compiler (FP32): 2 gives
// the register cap 128; the stage-2 pass (L_t only) runs 4 (cap 64; at most a
// few dozen bytes of spills for n_q <= 3), whose extra warps hide the latency
// of its face-moment reads (3-6 % faster than 3 CTAs at cap 80).  At n_q = 4
// (two warps per cell) every pass runs 3 (cap 80, no spills): 17-21 % faster
// than 2 at 128^3 P3; at n_q = 3 three CTAs made stage 1 slower (P3) or no
// faster (P2).
// CELL_PREFETCH: L2 prefetch of the next tile's face-moment blocks at stage 1
// (with a CTA barrier per tile it saved 2 %; with the decoupled tile loop it
// costs 0.8 %, so it is off)
#ifndef CELL_PREFETCH
#define CELL_PREFETCH 0
#endif
#ifndef CELL_MIN_CTAS_F32
#define CELL_MIN_CTAS_F32 2
#endif
template <class R, int NQ, int MODE>
constexpr int cell_min_ctas() {
  return sizeof(R) == 4 ? (MODE == 2 && NQ <= 3 ? 4 : (NQ == 4 ? 3 : CELL_MIN_CTAS_F32)) : 1;
}
template <class R, int ORDER, int NQ, int MODE, class Tin, class E = R>
__global__ void __launch_bounds__(CellLayout<ORDER, NQ>::WARPS * 32, (cell_min_ctas<R, NQ, MODE>()))
    k_cell(const Tin* __restrict__ Qin, const R* __restrict__ G, const StageIO<R, E> io, const GasPar<R> gp,
           const MeshDev m, const double dt, unsigned* __restrict__ flag) {
  using LY = CellLayout<ORDER, NQ>;
  using S = CellSmem<R, ORDER, NQ, Tin, E, MODE>;
  constexpr bool SPLIT = !std::is_same<E, R>::value;  // FP32 flux, FP64 epilogue
  constexpr int NM = LY::NM, NP = LY::NP, NC = S::NC, CB = LY::CB, PG = LY::PG, GW = LY::GW, NT = n_tmodes(ORDER);
  constexpr int NOUT = LY::NOUT, NOP = LY::NOP, NMP = S::NMP, NCP = S::NCP;
  using CBs = CellBasis<R, ORDER, NQ>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* const bt = reinterpret_cast<R*>(smem_raw + S::bt_off);  // [NP][BW] basis table
  R(*red)[GW][2][NOP] = reinterpret_cast<R(*)[GW][2][NOP]>(smem_raw + S::red_off);  // GW > 1 only
  int4* dsc = reinterpret_cast<int4*>(smem_raw + S::tab_off);  // [NC] face-block offsets of output v NM + n
  R(*dsg)[4] = reinterpret_cast<R(*)[4]>(dsc + NC);            // [NC] their parity signs
  E* invM = reinterpret_cast<E*>(dsg + NC);
  int* tix = reinterpret_cast<int*>(invM + NM);  // [3][NM] tangential index, then [3][NM] parity sign
  const int tid = threadIdx.x, nthr = LY::WARPS * 32;
  const int lane = tid & 31, lg = lane % PG, warp = tid >> 5;
  const int cb = GW == 1 ? warp * LY::CPW + lane / PG : warp / GW;  // cell of this lane within the CTA
  const int gw = GW == 1 ? 0 : warp % GW;                            // which warp of the cell
  const int pidx = gw * 32 + lg;                                      // Gauss point of this lane
  const int nx = m.nx, ny = m.ny, nz = m.nz;
  const long long nc = m.ncell;

  for (int e = tid; e < NM; e += nthr) {
    // (2a+1)(2b+1)(2c+1) / |K|; on a rectilinear mesh the 1/|K| of each cell
    // is applied in the epilogue
    invM[e] = (E)((2 * mode_exp(e, 0) + 1) * (2 * mode_exp(e, 1) + 1) * (2 * mode_exp(e, 2) + 1)) *
              (mesh_nonuniform(m) ? E(1) : mesh_ivol<E>(m));
#pragma unroll
    for (int D = 0; D < 3; ++D) {
      tix[D * NM + e] = tmode_index(mode_exp(e, tan1(D)), mode_exp(e, tan2(D)));
      tix[3 * NM + D * NM + e] = (mode_exp(e, D) % 2 == 0) ? 1 : -1;
    }
  }
  // (the descriptors serve the persistent one-cell-per-warp layout only; at
  // n_q = 4 every CTA handles one tile and would rebuild them for nothing)
  for (int e = tid; GW == 1 && e < NC; e += nthr) {
    const int v = e / NM, n = e % NM;
    int off[3];
  #pragma unroll
    for (int D = 0; D < 3; ++D) {
      off[D] = v * NT + tmode_index(mode_exp(n, tan1(D)), mode_exp(n, tan2(D)));
      dsg[e][D] = (mode_exp(n, D) % 2 == 0) ? R(1) : R(-1);
    }
    dsc[e] = make_int4(off[0], off[1], off[2], n);
    dsg[e][3] = R(0);
  }
  // basis table (persistent layout, k <= 2): one row per point
  for (int p = tid; S::TABLE && p < NP; p += nthr) {
    const CBs cbas(p);
    R* const rw = bt + p * CBs::BW;
  #pragma unroll
    for (int mm = 0; mm < NM; ++mm) {
      rw[CBs::POFF + mm] = cbas.phi(mm);
  #pragma unroll
      for (int d = 0; d < 3; ++d)
        if (mode_exp(mm, d) > 0) rw[CBs::gslot(mm, d)] = cbas.grad(mm, d);
    }
    rw[CBs::WOFF] = cbas.w;
  }

  const E h = (E)dt, h2 = (E)(dt * dt);
  // Everything after the staging of one tile (CB consecutive cells along x of
  // row (j, k)), reading the coefficients from coef[NC][CB].  With GW = 1 the
  // results go to so[kind][NC][CB] in shared memory (written out by flush).
  auto tile = [&](const int i0, const int j, const int k, const R (*coef)[NCP], E (*so)[NC][CB]) {
    const size_t row = ((size_t)k * ny + j) * nx;
    // ---- interior flux of Eq. (flux-2) at this lane's Gauss point ----
    // Every lane evaluates a physical state: spare lanes take point 0 and
    // cells beyond the row end hold a copy of a cell of the row (staged so),
    // so the flux is finite everywhere and a zero weight removes what is not
    // this cell's.
    const bool active = (pidx < NP) && (i0 + cb < nx);
    const int pp = pidx < NP ? pidx : 0;
    const R* const brow = bt + pp * CBs::BW;  // this point's basis row (table layout)
    const CBs lbas(pp);                       // the basis in registers otherwise
    const int icell = (i0 + cb < nx) ? i0 + cb : nx - 1;
    const R sc[3] = {cell_sc<R>(m, 0, icell), cell_sc<R>(m, 1, j), cell_sc<R>(m, 2, k)};
    const R cvol = mesh_nonuniform(m) ? cell_w<R>(m, 0, icell) * cell_w<R>(m, 1, j) * cell_w<R>(m, 2, k) : mesh_vol<R>(m);
    R Fw[3][5], Ftw[3][5];  // w |K| (2/h_d) F_d, same for F_t
    {
      // Q_h and its reference gradients at the point (each variable's
      // coefficients read four modes at a time with 16-byte loads)
      R br[S::TABLE ? CBs::WOFF : 4];
      if constexpr (S::TABLE) lds16<CBs::WOFF>(brow, br);
      auto phi = [&](int mm) {
        if constexpr (S::TABLE) return br[CBs::POFF + mm];
        else return lbas.phi(mm);
      };
      auto gph = [&](int mm, int d) {
        if constexpr (S::TABLE) return br[CBs::gslot(mm, d)];
        else return lbas.grad(mm, d);
      };
      R q[5], dq[3][5];
  #pragma unroll
      for (int v = 0; v < 5; ++v) {
        R s0 = R(0), g0 = R(0), g1 = R(0), g2 = R(0);
  #pragma unroll
        for (int c0 = 0; c0 < NM; c0 += 4) {
          R cv[4];
          lds16<4>(&coef[cb][v * NMP + c0], cv);
  #pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int mm = c0 + u;
            if (mm < NM) {
              s0 += cv[u] * phi(mm);
              // P'_0 = 0: modes constant along an axis have no gradient term there
              if (mode_exp(mm, 0) > 0) g0 += cv[u] * gph(mm, 0);
              if (mode_exp(mm, 1) > 0) g1 += cv[u] * gph(mm, 1);
              if (mode_exp(mm, 2) > 0) g2 += cv[u] * gph(mm, 2);
            }
          }
        }
        q[v] = s0;
        dq[0][v] = g0 * sc[0];
        dq[1][v] = g1 * sc[1];
        dq[2][v] = g2 * sc[2];
      }
      R F[3][5], Ft[3][5];
      const bool ok = interior_flux(q, dq, gp, F, Ft);
      if (active && !ok) atomicOr(flag, 1u);
      const R w = active ? (S::TABLE ? brow[CBs::WOFF] : lbas.w) * cvol : R(0);
  #pragma unroll
      for (int d = 0; d < 3; ++d)
  #pragma unroll
        for (int v = 0; v < 5; ++v) {
          Fw[d][v] = w * sc[d] * F[d][v];
          Ftw[d][v] = w * sc[d] * Ft[d][v];
        }
    }

    // One cell per warp: the face-moment blocks of this lane's cell, its low
    // faces normal to D = 0, 1, 2 (fb[D]) and its high neighbours' (fb[3 + D]),
    // addressed once per tile.
    const R* fb[6];
    if constexpr (GW == 1) {
      const int ic = i0 + cb < nx ? i0 + cb : nx - 1;
      const size_t cell = row + ic;
      const size_t up[3] = {row + wrapm(ic + 1, nx), ((size_t)k * ny + wrapm(j + 1, ny)) * nx + ic,
                            ((size_t)wrapm(k + 1, nz) * ny + j) * nx + ic};
  #pragma unroll
      for (int D = 0; D < 3; ++D) {
        fb[D] = G + ((size_t)D * nc + cell) * (10 * NT);
        fb[3 + D] = G + ((size_t)D * nc + up[D]) * (10 * NT);
      }
    }

    // One output (variable v, mode n) of the cell at x index i: the six faces'
    // moments with the sign/parity of Eq. (operator) added to the volume sums
    // (the assembly of R, R_t, part of the projection: in the flux precision
    // R), then M^-1 and the stage epilogue in the precision E; with E = R the
    // accumulation into the stored FP64 state is the one FP64 operation.
    // SPLIT: the mode-0 outputs (the cell averages, whose totals the scheme
    // conserves) sum their FP32 face moments exactly (ExactAcc); each face
    // enters its two cells with opposite signs, so the totals hold to FP64
    // rounding.
    auto finish = [&](int v, int n, int i, int cc, R sF_, R sT_) {
      const size_t cell = row + i;
      const size_t idx = (size_t)(v * NM + n) * nc + cell;
      E sF, sT;
      auto assemble = [&](auto aF, auto aT) {
        if constexpr (GW == 1) {
          const int o = v * NM + n;
          const int4 ds = dsc[o];
          const int dof[3] = {ds.x, ds.y, ds.z};
          R sg[3];
          if constexpr (sizeof(R) == 4) {
            const float4 q = *reinterpret_cast<const float4*>(dsg[o]);
            sg[0] = q.x, sg[1] = q.y, sg[2] = q.z;
          } else {
            const double2 q0 = reinterpret_cast<const double2*>(dsg[o])[0];
            sg[0] = q0.x, sg[1] = q0.y, sg[2] = dsg[o][2];
          }
  #pragma unroll
          for (int D = 0; D < 3; ++D) {
            const R* lo = fb[D] + dof[D];
            const R* hi = fb[3 + D] + dof[D];
            aF.add(sg[D], lo[0], hi[0]);
            aT.add(sg[D], lo[5 * NT], hi[5 * NT]);
          }
        } else {
  #pragma unroll
          for (int D = 0; D < 3; ++D) {
            const int t = tix[D * NM + n];
            const R sg = (R)tix[3 * NM + D * NM + n];
            size_t up;
            if (D == 0)
              up = row + wrapm(i + 1, nx);
            else if (D == 1)
              up = ((size_t)k * ny + wrapm(j + 1, ny)) * nx + i;
            else
              up = ((size_t)wrapm(k + 1, nz) * ny + j) * nx + i;
            const R* gD = G + (size_t)D * nc * (10 * NT) + v * NT + t;  // face-major: [D][face][10][NT]
            aF.add(sg, gD[cell * (10 * NT)], gD[up * (10 * NT)]);
            aT.add(sg, gD[cell * (10 * NT) + 5 * NT], gD[up * (10 * NT) + 5 * NT]);
          }
        }
        sF = aF.template get<E>();
        sT = aT.template get<E>();
      };
      if constexpr (SPLIT) {
        if (n == 0)
          assemble(ExactAcc(sF_), ExactAcc(sT_));
        else
          assemble(PlainAcc<R>(sF_), PlainAcc<R>(sT_));
      } else {
        assemble(PlainAcc<R>(sF_), PlainAcc<R>(sT_));
      }
      E iM = invM[n];
      if (mesh_nonuniform(m))  // 1/|K| = (2/h_x)(2/h_y)(2/h_z) / 8
        iM *= cell_sc<E>(m, 0, i) * cell_sc<E>(m, 1, j) * cell_sc<E>(m, 2, k) * E(0.125);
      const E Lv = sF * iM, Ltv = sT * iM;
      if constexpr (GW == 1) {
        const int o = v * NM + n;
        if (MODE == MODE_RESIDUAL) {
          so[0][o][cc] = Lv;
          so[1][o][cc] = Ltv;
        } else if (MODE == MODE_STAGE1) {
          if constexpr (SPLIT)  // the increment of Q* only; flush adds it to the FP64 state
            so[0][o][cc] = E(0.5) * h * Lv + (h2 * E(0.125)) * Ltv;
          else
            so[0][o][cc] = coef[cc][v * NMP + n] + (R(0.5) * h * Lv + (h2 * R(0.125)) * Ltv);
          so[1][o][cc] = h * Lv + (h2 * E(1.0 / 6.0)) * Ltv;
        } else {
          so[0][o][cc] = Ltv;
        }
      } else if (MODE == MODE_RESIDUAL) {
        io.L[idx] = (double)Lv;
        io.Lt[idx] = (double)Ltv;
      } else if (MODE == MODE_STAGE1) {
        if constexpr (SPLIT)
          io.Qs[idx] = (R)(io.Qn[idx] + (E(0.5) * h * Lv + (h2 * E(0.125)) * Ltv));
        else
          io.Qs[idx] = coef[cc][v * NMP + n] + (R(0.5) * h * Lv + (h2 * R(0.125)) * Ltv);
        io.inc[idx] = h * Lv + (h2 * E(1.0 / 6.0)) * Ltv;
      } else {
        const double q = io.Qn[idx] + (double)(io.inc[idx] + (h2 * E(1.0 / 3.0)) * Ltv);
        io.Qn[idx] = q;
        if (io.Qf) io.Qf[idx] = (R)q;
      }
    };
    // this lane's contribution to output o (v = o / NM, mode n = o % NM; mode
    // 0 has no volume term), with the basis gradients at its point
    R gr[S::TABLE ? CBs::POFF : 4];
    if constexpr (S::TABLE) lds16<CBs::POFF>(brow, gr);
    auto gvol = [&](int n, int d) {
      if constexpr (S::TABLE) return gr[CBs::gslot(n, d)];
      else return lbas.grad(n, d);
    };
    auto vol_term = [&](const R(&Fk)[3][5], int o) {
      R c = R(0);
      if (o < 5 * NM) {
        const int v = o / NM, n = o % NM;
        if (mode_exp(n, 0) > 0) c += Fk[0][v] * gvol(n, 0);
        if (mode_exp(n, 1) > 0) c += Fk[1][v] * gvol(n, 1);
        if (mode_exp(n, 2) > 0) c += Fk[2][v] * gvol(n, 2);
      }
      return c;
    };

    if constexpr (GW == 1) {
      // ---- volume projection fused with the epilogue: the volume outputs
      // (modes n >= 1, j = v (NM-1) + n-1) are summed over the cell's lanes a
      // block at a time, after which lane lg holds output j of both kinds (F
      // and F_t) and finishes it; the five mode-0 outputs have face terms
      // only.  No cross-warp exchange, no CTA barrier. ----
      constexpr int NV = 5 * (NM - 1);
      const bool live = i0 + cb < nx;
      auto vslot = [&](const R(&Fk)[3][5], int j) {
        return j < NV ? vol_term(Fk, (j / (NM - 1)) * NM + 1 + j % (NM - 1)) : R(0);
      };
      if constexpr (PG == 32) {
        // one cell per warp: for each block of 32 outputs every lane with a
        // Gauss point writes its contributions as one shared-memory row, and
        // lane lg sums column lg over the cell's points in a fixed order
        // (packed FP32 pairs: F and F_t of one output side by side).  No
        // shuffles and no lane-dependent selects.
        constexpr int NBLK = (NV + 31) / 32, RM = NV - (NBLK - 1) * 32;
        constexpr bool M0_LAST = RM + 5 <= 32;  // mode 0 on the idle lanes of the last pass
        constexpr bool TWO = MODE != MODE_STAGE2;
        constexpr int TS = S::TS;
        R* const trows = reinterpret_cast<R*>(smem_raw + S::tr_off) + (size_t)warp * NP * TS;
  #pragma unroll
        for (int blk = 0; blk < NBLK; ++blk) {
          const int nsl = blk == NBLK - 1 ? RM : 32;  // output slots of this block
          if (pidx < NP) {
            R* const row = trows + pidx * TS;
            if constexpr (TWO && sizeof(R) == 4) {
  #pragma unroll
              for (int q = 0; q < 16; ++q)
                if (2 * q < nsl)
                  reinterpret_cast<float4*>(row)[q] =
                      make_float4(vslot(Fw, blk * 32 + 2 * q), vslot(Ftw, blk * 32 + 2 * q),
                                  vslot(Fw, blk * 32 + 2 * q + 1), vslot(Ftw, blk * 32 + 2 * q + 1));
            } else if constexpr (TWO) {
  #pragma unroll
              for (int q = 0; q < 32; ++q)
                if (q < nsl)
                  reinterpret_cast<double2*>(row)[q] = make_double2(vslot(Fw, blk * 32 + q), vslot(Ftw, blk * 32 + q));
            } else if constexpr (sizeof(R) == 4) {
  #pragma unroll
              for (int q = 0; q < 8; ++q)
                if (4 * q < nsl)
                  reinterpret_cast<float4*>(row)[q] =
                      make_float4(vslot(Ftw, blk * 32 + 4 * q), vslot(Ftw, blk * 32 + 4 * q + 1),
                                  vslot(Ftw, blk * 32 + 4 * q + 2), vslot(Ftw, blk * 32 + 4 * q + 3));
            } else {
  #pragma unroll
              for (int q = 0; q < 16; ++q)
                if (2 * q < nsl)
                  reinterpret_cast<double2*>(row)[q] =
                      make_double2(vslot(Ftw, blk * 32 + 2 * q), vslot(Ftw, blk * 32 + 2 * q + 1));
            }
          }
          __syncwarp();
          // NQ partial sums, one per plane of points (the rows L = a NQ^2 + ...
          // of one a), then combined in order: NQ independent add chains
          R sF = R(0), sT = R(0);
          if constexpr (TWO && sizeof(R) == 4) {
            float2 acc[NQ];
  #pragma unroll
            for (int a = 0; a < NQ; ++a) {
              acc[a] = reinterpret_cast<const float2*>(trows + a * NQ * NQ * TS)[lg];
  #pragma unroll
              for (int L = a * NQ * NQ + 1; L < (a + 1) * NQ * NQ; ++L)
                acc[a] = __fadd2_rn(acc[a], reinterpret_cast<const float2*>(trows + L * TS)[lg]);
            }
  #pragma unroll
            for (int a = 1; a < NQ; ++a) acc[0] = __fadd2_rn(acc[0], acc[a]);
            sF = acc[0].x;
            sT = acc[0].y;
          } else if constexpr (TWO) {
            R aF[NQ], aT[NQ];
  #pragma unroll
            for (int a = 0; a < NQ; ++a) {
              aF[a] = aT[a] = R(0);
  #pragma unroll
              for (int L = a * NQ * NQ; L < (a + 1) * NQ * NQ; ++L) {
                const double2 x = reinterpret_cast<const double2*>(trows + L * TS)[lg];
                aF[a] += x.x;
                aT[a] += x.y;
              }
            }
  #pragma unroll
            for (int a = 0; a < NQ; ++a) {
              sF += aF[a];
              sT += aT[a];
            }
          } else {
            R aT[NQ];
  #pragma unroll
            for (int a = 0; a < NQ; ++a) {
              aT[a] = trows[a * NQ * NQ * TS + lg];
  #pragma unroll
              for (int L = a * NQ * NQ + 1; L < (a + 1) * NQ * NQ; ++L) aT[a] += trows[L * TS + lg];
            }
  #pragma unroll
            for (int a = 0; a < NQ; ++a) sT = a ? sT + aT[a] : aT[0];
          }
          __syncwarp();  // the rows are rewritten by the next block
          // one finish per lane and pass: output blk 32 + lg of the pass, else
          // (last pass) mode-0 output lg - RM
          int jo = blk * 32 + lg;
          int v = jo / (NM - 1), n = 1 + jo % (NM - 1);
          bool act = jo < NV;
          if (!act && blk == NBLK - 1 && M0_LAST && lg < RM + 5) {
            v = lg - RM;
            n = 0;
            sF = sT = R(0);
            act = true;
          }
          if (act && live) finish(v, n, i0 + cb, cb, sF, sT);
        }
        if constexpr (!M0_LAST) {
          if (lg >= 32 - 5 && live) finish(lg - (32 - 5), 0, i0 + cb, cb, R(0), R(0));
        }
      } else {
      // ---- several cells per warp (n_q = 2): the PG lanes of a cell reduce
      // PG volume outputs (modes n >= 1, j = v (NM-1) + n-1) at a time by a
      // butterfly, after which lane lg holds output j = blk PG + lg of both
      // kinds (F and F_t) and finishes it.  When the last block of RM outputs
      // fits twice into PG slots, its F and F_t sums share one butterfly (F in
      // slots 0..RM-1, F_t in RM..2RM-1) and a shuffle pairs them.  The five
      // mode-0 outputs have face terms only. ----
      constexpr int NB = NV / PG, RM = NV % PG;
      constexpr bool PACK = MODE != MODE_STAGE2 && RM > 0 && 2 * RM <= PG;
      constexpr int NBLK = NB + ((RM > 0 && !PACK) ? 1 : 0);
      constexpr bool M0_LAST = RM > 0 && RM + 5 <= PG;  // mode 0 on the idle lanes of the last pass
      // one finish per lane and pass: output j < NV of the pass, else (last
      // pass) mode-0 output lg - RM
      auto finish_pass = [&](int j, bool last, R sF, R sT) {
        int v = j / (NM - 1), n = 1 + j % (NM - 1);
        bool act = j < NV;
        if (!act && last && M0_LAST && lg < RM + 5) {
          v = lg - RM;
          n = 0;
          sF = sT = R(0);
          act = true;
        }
        if (act && live) finish(v, n, i0 + cb, cb, sF, sT);
      };
  #pragma unroll
      for (int blk = 0; blk < NBLK; ++blk) {
        R vF[PG], vT[PG];
  #pragma unroll
        for (int oo = 0; oo < PG; ++oo) {
          vF[oo] = vslot(Fw, blk * PG + oo);
          vT[oo] = vslot(Ftw, blk * PG + oo);
        }
        R oF[1], oT[1];
        group_reduce<PG, PG>(vF, oF, lg);
        group_reduce<PG, PG>(vT, oT, lg);
        finish_pass(blk * PG + lg, !PACK && blk == NBLK - 1, oF[0], oT[0]);
      }
      if constexpr (PACK) {
        R vv[PG];
  #pragma unroll
        for (int oo = 0; oo < PG; ++oo)
          vv[oo] = oo < RM ? vslot(Fw, NB * PG + oo) : (oo < 2 * RM ? vslot(Ftw, NB * PG + oo - RM) : R(0));
        R o1[1];
        group_reduce<PG, PG>(vv, o1, lg);
        const R oT = __shfl_down_sync(0xffffffffu, o1[0], RM);  // lane lg < RM: F_t sum from lane lg + RM
        finish_pass(lg < RM ? NB * PG + lg : NV, true, o1[0], oT);
      }
      if constexpr (!M0_LAST) {
        if (lg >= PG - 5 && live) finish(lg - (PG - 5), 0, i0 + cb, cb, R(0), R(0));
      }
      }
    } else {
      // ---- a cell spans GW warps: per-warp butterflies over the modes n >= 1,
      // partial sums through shared memory, then the epilogue over the CTA
      // (the stage-2 pass reduces the F_t kind only) ----
  #pragma unroll
      for (int kind = MODE == MODE_STAGE2 ? 1 : 0; kind < 2; ++kind) {
  #pragma unroll
        for (int c0 = 0; c0 < NOP; c0 += PG) {
          R val[PG];
  #pragma unroll
          for (int oo = 0; oo < PG; ++oo) {
            const int o = c0 + oo;  // v = o / (NM - 1), n = 1 + o % (NM - 1)
            val[oo] = o < NOUT ? vol_term(kind == 0 ? Fw : Ftw, (o / (NM - 1)) * NM + 1 + o % (NM - 1)) : R(0);
          }
          R outv[1];
          group_reduce<PG, PG>(val, outv, lg);
          red[cb][gw][kind][c0 + lg] = outv[0];
        }
      }
      __syncthreads();
      for (int o = tid; o < CB * NC; o += nthr) {
        const int cc = o % CB, rest = o / CB, mm = rest % NM, v = rest / NM;
        if (i0 + cc >= nx) continue;
        R sF = R(0), sT = R(0);
        if (mm > 0)
  #pragma unroll
          for (int g = 0; g < GW; ++g) {
            sF += red[cc][g][0][v * (NM - 1) + mm - 1];
            sT += red[cc][g][1][v * (NM - 1) + mm - 1];
          }
        finish(v, mm, i0 + cc, cc, sF, sT);
      }
    }
  };

  if constexpr (GW == 1) {
    // Persistent CTAs over the tiles; the coefficients of the next tile are
    // copied global -> shared with cp.async while the current tile is
    // computed.  Three buffers of staged coefficients, four of outputs, and
    // mbarriers in place of a CTA barrier per tile let a warp run up to one
    // tile ahead of the slowest warp of its CTA: in its n-th tile a thread
    //   waits full[n]  (tile n staged),
    //   waits done[n-2] (every warp finished tile n-2: its outputs complete,
    //                    its coefficient buffer free, and the outputs of tile
    //                    n-4, which every thread wrote out before computing
    //                    tile n-2, no longer needed), then stages tile n+1
    //                    into that coefficient buffer and writes tile n-2's
    //                    outputs out,
    //   computes tile n into output buffer n mod 4 and arrives done[n]
    // (coefficient buffers and barriers n mod 3; the phase of a barrier's
    // k-th use is k & 1).
    Tin(*raw)[CB][NCP] = reinterpret_cast<Tin(*)[CB][NCP]>(smem_raw);  // [buffer][cell][v NMP + n]
    R(*cvt)[NCP] = reinterpret_cast<R(*)[NCP]>(smem_raw + S::cvt_off);  // converted copy (Tin != R)
    // tile t = (k ny + j) ntx + tx, coordinates computed once per tile in 32
    // bits (the host keeps the tile count below 2^31)
    struct TileAt {
      int i0, j, k;
      size_t row;  // (k ny + j) nx
    };
    const unsigned ntx = (unsigned)(nx + CB - 1) / CB, ntiles = ntx * (unsigned)ny * (unsigned)nz;
    auto at = [&](unsigned t) {
      TileAt a;
      const unsigned r = t / ntx;
      a.i0 = (int)(t - r * ntx) * CB;
      a.j = (int)(r % (unsigned)ny);
      a.k = (int)(r / (unsigned)ny);
      a.row = (size_t)r * nx;
      return a;
    };
    // the tile gridDim.x further on, without per-tile divisions: tx advances
    // by the remainder gr of gridDim.x / ntx, the row index k ny + j by the
    // quotient gq (+1 on a carry); j wraps into k only when it passes ny
    const unsigned gq = gridDim.x / ntx, gr = gridDim.x - gq * ntx;
    auto next_at = [&](const TileAt& a) {
      TileAt n;
      unsigned tx = (unsigned)a.i0 / CB + gr, dr = gq;
      if (tx >= ntx) {
        tx -= ntx;
        ++dr;
      }
      unsigned jj = (unsigned)a.j + dr, kk = (unsigned)a.k;
      if (jj >= (unsigned)ny) {
        kk += jj / (unsigned)ny;
        jj %= (unsigned)ny;
      }
      n.i0 = (int)tx * CB;
      n.j = (int)jj;
      n.k = (int)kk;
      n.row = ((size_t)kk * ny + jj) * nx;
      return n;
    };
    // (cells beyond the row end get a copy of the row's first cell: every
    // lane's flux input stays physical)
    auto issue = [&](const TileAt& a, int b) {
      for (int e = tid; e < NC * CB; e += nthr) {
        const int cc = e % CB, comp = e / CB, i = a.i0 + cc;
        cp_async_zfill(&raw[b][cc][(comp / NM) * NMP + comp % NM], Qin + (size_t)comp * nc + a.row + (i < nx ? i : 0),
                       true);
      }
      cp_async_commit();
    };
    // outputs of a tile (in so[bb]) -> global memory, a row of CB consecutive
    // cells per (variable, mode): whole sectors instead of one value per row
    E(*so)[S::NKO][NC][CB] = reinterpret_cast<E(*)[S::NKO][NC][CB]>(smem_raw + S::out_off);
    auto flush = [&](const TileAt& a, int bb) {
      for (int e = tid; e < NC * CB; e += nthr) {
        const int cc = e % CB, o = e / CB, i = a.i0 + cc;
        if (i >= nx) continue;
        const size_t idx = (size_t)o * nc + a.row + i;
        if constexpr (MODE == MODE_RESIDUAL) {
          io.L[idx] = (double)so[bb][0][o][cc];
          io.Lt[idx] = (double)so[bb][S::NKO - 1][o][cc];
        } else if constexpr (MODE == MODE_STAGE1) {
          if constexpr (SPLIT)
            io.Qs[idx] = (R)(io.Qn[idx] + so[bb][0][o][cc]);
          else
            io.Qs[idx] = so[bb][0][o][cc];
          io.inc[idx] = so[bb][S::NKO - 1][o][cc];
        } else {
          const double q = io.Qn[idx] + (double)(io.inc[idx] + (h2 * E(1.0 / 3.0)) * so[bb][0][o][cc]);
          io.Qn[idx] = q;
          if (io.Qf) io.Qf[idx] = (R)q;
        }
      }
    };
    // L2 prefetch of the face-moment blocks a tile's epilogue reads (its cells'
    // low faces along x, y, z and the high neighbours'), one tile ahead: they
    // were written by the face kernels long before and are no longer in L2.
    // (Stage 2 reads only their F_t halves, and ran slower with it; used only
    // when CELL_PREFETCH is set.)
    auto prefetch_faces = [&](const TileAt& a) {
      constexpr int LINES = (10 * NT * (int)sizeof(R) + 127) / 128;  // 128-byte lines per face block
      for (int e = tid; e < (5 * CB + 1) * LINES; e += nthr) {
        const int sl = e / LINES, ln = e % LINES;
        int D, s, hi;
        if (sl <= CB) {
          D = 0, s = sl, hi = 0;
        } else if (sl <= 3 * CB) {
          D = 1, s = (sl - CB - 1) % CB, hi = (sl - CB - 1) / CB;
        } else {
          D = 2, s = (sl - 3 * CB - 1) % CB, hi = (sl - 3 * CB - 1) / CB;
        }
        int i = a.i0 + s;
        if (i >= nx) i -= nx;
        if (i >= nx) continue;
        const int cj = (D == 1 && hi) ? wrapm(a.j + 1, ny) : a.j, ck = (D == 2 && hi) ? wrapm(a.k + 1, nz) : a.k;
        const R* pf = G + ((size_t)D * nc + ((size_t)ck * ny + cj) * nx + i) * (10 * NT) + ln * (128 / sizeof(R));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
      }
    };
    if constexpr (S::DECOUPLED) {
      unsigned long long* const bar = reinterpret_cast<unsigned long long*>(smem_raw + S::bar_off);
      unsigned long long *const full = bar, *const done = bar + S::NBUF;
      if (tid == 0)
        for (int q = 0; q < 2 * S::NBUF; ++q) mbar_init(bar + q, nthr);
      __syncthreads();  // (the tables above and the barriers' initialisation)
      unsigned t = blockIdx.x;
      TileAt cur = at(t), p1 = cur, p2 = cur;  // tiles n, n - 1, n - 2
      if (t < ntiles) {
        issue(cur, 0);
        cp_async_mbar_arrive(&full[0]);
      }
      bool ok = true;
      unsigned n = 0;
      for (; t < ntiles; t += gridDim.x, ++n) {
        const int x = (int)(n % 3), xm2 = (int)((n + 1) % 3);  // n, n - 2 mod 3
        ok = mbar_wait(&full[x], (n / 3) & 1);
        if (ok && n >= 2) ok = mbar_wait(&done[xm2], ((n - 2) / 3) & 1);
        if (!ok) break;
        const unsigned tn = t + gridDim.x;
        TileAt nxt = cur;
        if (tn < ntiles) {
          nxt = next_at(cur);
          issue(nxt, xm2);
          cp_async_mbar_arrive(&full[xm2]);
          if (MODE != MODE_STAGE2 && CELL_PREFETCH) prefetch_faces(nxt);
        }
        if (n >= 2) flush(p2, (int)((n - 2) % 4));
        const R(*coef)[NCP];
        if constexpr (std::is_same<Tin, R>::value) {
          coef = raw[x];
        } else {
          // each warp converts its own cells (the only ones it reads; padding
          // included, so that the 16-byte loads read defined values)
          for (int e = lane; e < NCP * LY::CPW; e += 32) {
            const int cc = warp * LY::CPW + e / NCP, c = e % NCP;
            cvt[cc][c] = (R)raw[x][cc][c];
          }
          __syncwarp();
          coef = cvt;
        }
        tile(cur.i0, cur.j, cur.k, coef, so[n % 4]);
        mbar_arrive(&done[x]);
        p2 = p1;
        p1 = cur;
        cur = nxt;
      }
      // the last two tiles' outputs
      if (ok && n >= 2 && (ok = mbar_wait(&done[(n - 2) % 3], ((n - 2) / 3) & 1))) flush(p2, (int)((n - 2) % 4));
      if (ok && n >= 1 && (ok = mbar_wait(&done[(n - 1) % 3], ((n - 1) / 3) & 1))) flush(p1, (int)((n - 1) % 4));
      if (!ok) atomicOr(flag, 2u);
      cp_async_wait_all();
    } else {
      // stage 2 (F_t only): two buffers and one CTA barrier per tile (the
      // decoupled loop, CELL_DECOUPLE_STAGE2, ran this pass no faster)
      unsigned t = blockIdx.x;
      TileAt cur = at(t), prev = cur;
      bool have_prev = false;
      if (t < ntiles) issue(cur, 0);
      int b = 0;
      for (; t < ntiles; t += gridDim.x, b ^= 1) {
        cp_async_wait_all();
        __syncthreads();  // tile t staged by all threads; every warp is done with buffer b ^ 1
        const unsigned tn = t + gridDim.x;
        TileAt nxt = cur;
        if (tn < ntiles) {
          nxt = next_at(cur);
          issue(nxt, b ^ 1);
          if (MODE != MODE_STAGE2 && CELL_PREFETCH) prefetch_faces(nxt);
        }
        if (have_prev) flush(prev, b ^ 1);
        const R(*coef)[NCP];
        if constexpr (std::is_same<Tin, R>::value) {
          coef = raw[b];
        } else {
          // each warp converts its own cells (the only ones it reads; padding
          // included, so that the 16-byte loads read defined values)
          for (int e = lane; e < NCP * LY::CPW; e += 32) {
            const int cc = warp * LY::CPW + e / NCP, c = e % NCP;
            cvt[cc][c] = (R)raw[b][cc][c];
          }
          __syncwarp();
          coef = cvt;
        }
        tile(cur.i0, cur.j, cur.k, coef, so[b]);
        prev = cur;
        have_prev = true;
        cur = nxt;
      }
      __syncthreads();
      if (have_prev) flush(prev, b ^ 1);
    }
  } else {
    R(*coef)[NCP] = reinterpret_cast<R(*)[NCP]>(smem_raw + S::cvt_off);
    const int i0 = blockIdx.x * CB, j = blockIdx.y, k = blockIdx.z;
    const size_t row = ((size_t)k * ny + j) * nx;
    // (cells beyond the row end: a copy of the row's first cell; padding zero)
    for (int e = tid; e < NCP * CB; e += nthr) {
      const int cc = e / NCP, c = e % NCP, i = i0 + cc;
      coef[cc][c] = (c % NMP < NM) ? (R)__ldg(Qin + (size_t)((c / NMP) * NM + c % NMP) * nc + row + (i < nx ? i : 0))
                                   : R(0);
    }
    __syncthreads();
    tile(i0, j, k, coef, nullptr);
  }
}

// Launch geometry of k_cell: persistent CTAs (resident CTAs per SM x SMs, at
// most one per tile) when a cell fits in one warp, otherwise one CTA per tile.
// The persistent kernel strides over the tiles, so any grid size is correct;
// if the occupancy query fails, one CTA per tile is launched.
template <class R, int ORDER, int NQ, int MODE, class Tin, class E = R>
inline void cell_launch_config(const MeshDev& m, dim3& grid, size_t& smem) {
  using LY = CellLayout<ORDER, NQ>;
  smem = CellSmem<R, ORDER, NQ, Tin, E, MODE>::bytes;
  const long long ntx = (m.nx + LY::CB - 1) / LY::CB;
  if (LY::GW != 1) {
    grid = dim3((unsigned)ntx, (unsigned)m.ny, (unsigned)m.nz);
    return;
  }
  const long long ntiles = ntx * m.ny * m.nz;
  long long g = ntiles < 0x7fffffffLL ? ntiles : 0x7fffffffLL;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cell<R, ORDER, NQ, MODE, Tin, E>, LY::WARPS * 32, smem) ==
          cudaSuccess &&
      sms > 0 && per > 0 && (long long)sms * per < g)
    g = (long long)sms * per;
  grid = dim3((unsigned)g);
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
__global__ void __launch_bounds__(RED_THREADS) k_totals_part(const double* __restrict__ Q, const MeshDev m,
                                                             double* __restrict__ part) {
  const long long nc = m.ncell;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < nc; c += (long long)gridDim.x * RED_THREADS) {
    const double wc = cell_weight(m, c);
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += wc * Q[(size_t)(v * NM) * nc + c];
  }
  block_reduce_store<5>(acc, part);
}

// Values at the NQ^3 tensor Gauss points of a modal polynomial (coefficients
// co, the P_k Legendre basis) by sum factorisation: contract x, then y, then z
// (q[i][j][k] at (x_i, y_j, z_k)); zero and unit basis factors fold away.
template <int ORDER, int NQ>
__device__ __forceinline__ void tensor_points(const double (&co)[n_modes(ORDER)], double (&q)[NQ][NQ][NQ]) {
  constexpr int NM = n_modes(ORDER);
  double t1[ORDER + 1][ORDER + 1][NQ];  // [b][c][i]: sum over a
#pragma unroll
  for (int b = 0; b <= ORDER; ++b)
#pragma unroll
    for (int c = 0; c <= ORDER; ++c)
#pragma unroll
      for (int i = 0; i < NQ; ++i) t1[b][c][i] = 0.0;
#pragma unroll
  for (int mm = 0; mm < NM; ++mm)
#pragma unroll
    for (int i = 0; i < NQ; ++i)
      t1[mode_exp(mm, 1)][mode_exp(mm, 2)][i] += co[mm] * leg<double>(mode_exp(mm, 0), gauss_x(NQ, i));
  double t2[ORDER + 1][NQ][NQ];  // [c][i][j]: sum over b
#pragma unroll
  for (int c = 0; c <= ORDER; ++c)
#pragma unroll
    for (int i = 0; i < NQ; ++i)
#pragma unroll
      for (int j = 0; j < NQ; ++j) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b + c <= ORDER; ++b) s += t1[b][c][i] * leg<double>(b, gauss_x(NQ, j));
        t2[c][i][j] = s;
      }
#pragma unroll
  for (int i = 0; i < NQ; ++i)
#pragma unroll
    for (int j = 0; j < NQ; ++j)
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c <= ORDER; ++c) s += t2[c][i][j] * leg<double>(c, gauss_x(NQ, k));
        q[i][j][k] = s;
      }
}

// 1/x in FP64 for a density: FP32 reciprocal estimate refined by two
// Newton-Raphson steps r <- r + r (1 - x r) (quadratic convergence: the
// seed's 2^-23 relative error falls below FP64 rounding); outside the FP32
// normal range, the division.
__device__ __forceinline__ double recip64(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

template <int ORDER, int NQ>
__global__ void __launch_bounds__(RED_THREADS) k_ek_part(const double* __restrict__ Q, const MeshDev m,
                                                         double* __restrict__ part) {
  constexpr int NM = n_modes(ORDER);
  const long long nc = m.ncell;
  double acc[1] = {0};
  for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < nc; c += (long long)gridDim.x * RED_THREADS) {
    const double wc = cell_weight(m, c);
    double co[NM], rho[NQ][NQ][NQ], mom[NQ][NQ][NQ], m2[NQ][NQ][NQ];
#pragma unroll
    for (int mm = 0; mm < NM; ++mm) co[mm] = Q[(size_t)mm * nc + c];
    tensor_points<ORDER, NQ>(co, rho);
#pragma unroll
    for (int a = 0; a < NQ; ++a)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int cz = 0; cz < NQ; ++cz) m2[a][b][cz] = 0.0;
#pragma unroll
    for (int v = 1; v < 4; ++v) {
#pragma unroll
      for (int mm = 0; mm < NM; ++mm) co[mm] = Q[(size_t)(v * NM + mm) * nc + c];
      tensor_points<ORDER, NQ>(co, mom);
#pragma unroll
      for (int a = 0; a < NQ; ++a)
#pragma unroll
        for (int b = 0; b < NQ; ++b)
#pragma unroll
          for (int cz = 0; cz < NQ; ++cz) m2[a][b][cz] += mom[a][b][cz] * mom[a][b][cz];
    }
#pragma unroll
    for (int a = 0; a < NQ; ++a)
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int cz = 0; cz < NQ; ++cz)
          acc[0] += wc * (gauss_w(NQ, a) * gauss_w(NQ, b) * gauss_w(NQ, cz) * 0.5 * m2[a][b][cz] *
                          recip64(rho[a][b][cz]));
  }
  block_reduce_store<1>(acc, part);
}

// Enstrophy integral sum_cells sum_p w |K| rho |omega|^2 / 2 at the n_q^3
// cell points (Sec. 5.3): omega = curl U, grad U = (grad m - U grad rho)/rho.
template <int ORDER, int NQ>
__global__ void __launch_bounds__(RED_THREADS) k_enstrophy_part(const double* __restrict__ Q, const MeshDev m,
                                                                double* __restrict__ part) {
  constexpr int NM = n_modes(ORDER);
  const long long nc = m.ncell;
  double acc[1] = {0};
  for (long long c = (long long)blockIdx.x * RED_THREADS + threadIdx.x; c < nc; c += (long long)gridDim.x * RED_THREADS) {
    const double wc = cell_weight(m, c);
    const int ci[3] = {(int)(c % m.nx), (int)((c / m.nx) % m.ny), (int)(c / ((long long)m.nx * m.ny))};
    const double sc[3] = {cell_sc<double>(m, 0, ci[0]), cell_sc<double>(m, 1, ci[1]), cell_sc<double>(m, 2, ci[2])};
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
          const double x[3] = {gauss_x(NQ, a), gauss_x(NQ, b), gauss_x(NQ, cz)};
          double q[4] = {0, 0, 0, 0}, g[3][4] = {{0}};
#pragma unroll
          for (int mm = 0; mm < NM; ++mm) {
            const int e[3] = {mode_exp(mm, 0), mode_exp(mm, 1), mode_exp(mm, 2)};
            const double P[3] = {leg<double>(e[0], x[0]), leg<double>(e[1], x[1]), leg<double>(e[2], x[2])};
            const double dP[3] = {dleg<double>(e[0], x[0]), dleg<double>(e[1], x[1]), dleg<double>(e[2], x[2])};
            const double B = P[0] * P[1] * P[2];
            const double dB[3] = {dP[0] * P[1] * P[2], P[0] * dP[1] * P[2], P[0] * P[1] * dP[2]};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              q[v] += co[v][mm] * B;
#pragma unroll
              for (int d = 0; d < 3; ++d) g[d][v] += co[v][mm] * dB[d] * sc[d];
            }
          }
          const double ir = 1.0 / q[0];
          double du[3][3];  // du[d][i] = d U_i / d x_d
#pragma unroll
          for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int i = 0; i < 3; ++i) du[d][i] = (g[d][1 + i] - q[1 + i] * ir * g[d][0]) * ir;
          const double w0 = du[1][2] - du[2][1], w1 = du[2][0] - du[0][2], w2 = du[0][1] - du[1][0];
          acc[0] += wc * (gauss_w(NQ, a) * gauss_w(NQ, b) * gauss_w(NQ, cz) * 0.5 * q[0] * (w0 * w0 + w1 * w1 + w2 * w2));
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
