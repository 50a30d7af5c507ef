// Transposed residual Jacobian, fused into one stage of the Runge-Kutta discrete adjoint
// (section "Unsteady adjoint": the A_kji, A^v_kji, D_kjil terms; "Implementation":
// the adjoint of the discrete scheme; "Energy analysis": the added viscosity).
//
// For the face flux Phi = (F_L + F_R)/2 - F^v of ns_rhs.cu the transpose is gathered
// per cell c from quantities built per face f = (L, R) in direction d:
//   Fb   = (a_L - a_R) / dx_d                                (adjoint of F^v at f)
//   s_j  = Fb[1+j] + Fb[4] uf_j                              (adjoint of sigma_dj)
//   normal gradient adjoint  nb_k = mu s_k + [k = d] mu s_d / 3,  nb_e = alpha Fb[4]
//   face-velocity adjoint    ub_j = Fb[4] sigma_dj           (primal stress row d)
// The tangential gradient adjoints of a face only ever hit u_d (mu s_l) and u_l
// (-2/3 mu s_d) for l != d, so per cell it suffices to sum s over the two faces in
// each direction, S_d(c) = s(c - e_d/2) + s(c + e_d/2), and
//   T[k][l] = mu S_k[l] (k != l),   T[l][l] = -2/3 mu sum_{d != l} S_d[d]
//   ubar_k(c) += (T[k][l](c - e_l) - T[k][l](c + e_l)) / (4 dx_l).
// The convective part is sum_d A_d(w_c)^T (a(c+e_d) - a(c-e_d)) / (2 dx_d).  The sum of
// primitive adjoints is then pulled back to conservative variables.
//
// Epilogue: the four stage products are summed in the stage type (G = sum_i g_i) and
// only the last stage forms lam^n = lam^{n+1} + G in FP64 (one FP64 add per component
// and step); the next seed is Anext = cl lam^{n+1} + cg g + cs G (the G term carries the
// earlier stages' products that a tableau with two nonzero entries in a column needs,
// as SSP-RK3's first stage does); the seeds a_i are summed
// the same way for the source sensitivity.
#include <type_traits>

#include "ns_common.cuh"
#include "ns_kernels.h"
#include "ns_roe.cuh"

namespace ns {
namespace adjk {

// Tile of the adjoint stage kernel: TX x TY columns (one thread per column).
#ifndef NS_ADJ_TY
#define NS_ADJ_TY 8
#endif
constexpr int TY = NS_ADJ_TY;
constexpr int NT = TX * TY;
constexpr int SY = TY + 2;
constexpr int SP = SX * SY;

namespace {

// In-plane offsets, periodic wrap resolved, of this thread's two shared positions
// t = tid and t = tid + NT (the same in every plane of the CTA's range).
struct AdjHalo {
  int o[2];
};
__device__ __forceinline__ AdjHalo adj_halo(const GridDesc& g, int x0, int y0) {
  AdjHalo h;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int t = threadIdx.x + it * NT;
    const int ly = t / SX;
    const int lx = t - ly * SX;
    h.o[it] = t < SP ? wrap(y0 + ly - 1, g.ny) * g.nx + wrap(x0 + lx - 1, g.nx) : 0;
  }
  return h;
}

// Register-staged plane load (primal primitives, adjoint input and, with the added
// viscosity, nu) so that the next plane's global loads overlap the current plane's work.
static_assert(SP <= 2 * NT, "a plane must fit two load rounds");
template <class CT>
struct AdjPlaneRegs {
  CT q[2][5];
  CT a[2][5];
  CT n[2];
};

template <class CT, class TIN, class TA>
__device__ __forceinline__ void adj_plane_load(AdjPlaneRegs<CT>& r, const GridDesc& g, size_t boxoff, int b,
                                               int k, const AdjHalo& h, const TIN* __restrict__ W,
                                               const TA* __restrict__ A, double ca, const float* __restrict__ nu,
                                               const double* __restrict__ nud) {
  const int kz = wrap(k, g.nz);
  const size_t pb = boxoff + (size_t)kz * g.plane;
  const CT cac = CT(ca);
  const long long n1 = g.cells * g.batch, n5 = 5 * n1;   // field extents (debug bounds checks)
  (void)n1;
  (void)n5;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    if (threadIdx.x + it * NT < SP) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        r.q[it][v] = cvt<CT>(NS_LD(g, W, pb + v * (size_t)g.cells, h.o[it], n5));
        r.a[it][v] = cac * cvt<CT>(NS_LD(g, A, pb + v * (size_t)g.cells, h.o[it], n5));
      }
    }
  }
  if (nu) {
    const size_t nb = (size_t)b * g.cells + (size_t)kz * g.plane;
#pragma unroll
    for (int it = 0; it < 2; ++it)
      if (threadIdx.x + it * NT < SP) r.n[it] = CT(NS_LD(g, nu, nb, h.o[it], n1));
  } else if (nud) {
    const size_t nb = (size_t)b * g.cells + (size_t)kz * g.plane;
#pragma unroll
    for (int it = 0; it < 2; ++it)
      if (threadIdx.x + it * NT < SP) r.n[it] = cvt<CT>(NS_LD(g, nud, nb, h.o[it], n1));
  }
}

template <class CT>
__device__ __forceinline__ void adj_plane_store(const AdjPlaneRegs<CT>& r, CT* __restrict__ sq,
                                                CT* __restrict__ sa, CT* __restrict__ sn, bool with_nu) {
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int t = threadIdx.x + it * NT;
    if (t < SP) {
      const CT ir = CT(1) / r.q[it][0];
      const CT u0 = r.q[it][1] * ir, u1 = r.q[it][2] * ir, u2 = r.q[it][3] * ir;
      sq[0 * SP + t] = r.q[it][0];
      sq[1 * SP + t] = u0;
      sq[2 * SP + t] = u1;
      sq[3 * SP + t] = u2;
      sq[4 * SP + t] = r.q[it][4] * ir - CT(0.5) * (u0 * u0 + u1 * u1 + u2 * u2);
#pragma unroll
      for (int v = 0; v < 5; ++v) sa[v * SP + t] = r.a[it][v];
      if (with_nu) sn[t] = r.n[it];
    }
  }
}

// s-vector of the face between shared positions iL (slot of QL/AL) and iR.
template <int D, class CT>
__device__ __forceinline__ void face_s(const Coef<CT>& c, const CT* QL, const CT* AL, int iL,
                                       const CT* QR, const CT* AR, int iR, CT s[3], CT& fb4) {
  fb4 = (AL[4 * SP + iL] - AR[4 * SP + iR]) * c.idx[D];
  int j0 = 0;
  if constexpr (std::is_same<CT, float>::value) {
    // components 1 and 2 side by side in paired FP32 instructions
    const float2 fb = __fmul2_rn(sub2(f2(AL[SP + iL], AL[2 * SP + iL]), f2(AR[SP + iR], AR[2 * SP + iR])),
                                 f2(c.idx[D], c.idx[D]));
    const float2 uf = __fmul2_rn(f2(0.5f, 0.5f),
                                 __fadd2_rn(f2(QL[SP + iL], QL[2 * SP + iL]), f2(QR[SP + iR], QR[2 * SP + iR])));
    const float2 sv = __ffma2_rn(f2(fb4, fb4), uf, fb);
    s[0] = sv.x;
    s[1] = sv.y;
    j0 = 2;
  }
#pragma unroll
  for (int j = j0; j < 3; ++j) {
    const CT fb = (AL[(1 + j) * SP + iL] - AR[(1 + j) * SP + iR]) * c.idx[D];
    const CT uf = CT(0.5) * (QL[(1 + j) * SP + iL] + QR[(1 + j) * SP + iR]);
    s[j] = fb + fb4 * uf;
  }
}

// Primal stress row D at a face from the two cells' primitives and the tangential face
// gradients of (u1, u2, u3) along T1 = (D+1)%3, T2 = (D+2)%3.  Only gt1[D], gt2[D] (the
// cross terms) and gt1[T1], gt2[T2] (the divergence) are read.
template <int D, class CT>
__device__ __forceinline__ void face_stress(const Coef<CT>& c, const CT* qL, const CT* qR,
                                            const CT* gt1, const CT* gt2, CT sig[3]) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  CT g[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    g[k][D] = (qR[k] - qL[k]) * c.idx[D];
    g[k][T1] = gt1[k];
    g[k][T2] = gt2[k];
  }
  const CT div = g[0][0] + g[1][1] + g[2][2];
#pragma unroll
  for (int j = 0; j < 3; ++j) sig[j] = c.mu * (g[j][D] + g[D][j]);
  sig[D] = sig[D] - CT(2.0 / 3.0) * c.mu * div;
}

// 7-value packet of a face from its s-vector and Fb[4]: nb[0..2] (u), nb[3] (e), ub[0..2].
template <int D, class CT>
__device__ __forceinline__ void face_packet_s(const Coef<CT>& c, const CT s[3], CT fb4, const CT* QL,
                                              int iL, const CT* QR, int iR, const CT* gt1,
                                              const CT* gt2, CT pk[7]) {
  CT uL[3], uR[3], sig[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    uL[j] = QL[(1 + j) * SP + iL];
    uR[j] = QR[(1 + j) * SP + iR];
  }
  face_stress<D>(c, uL, uR, gt1, gt2, sig);
#pragma unroll
  for (int k = 0; k < 3; ++k) pk[k] = c.mu * s[k];
  pk[D] = pk[D] + CT(1.0 / 3.0) * c.mu * s[D];
  pk[3] = c.alpha * fb4;
#pragma unroll
  for (int j = 0; j < 3; ++j) pk[4 + j] = fb4 * sig[j];
}

template <int D, class CT>
__device__ __forceinline__ void face_packet(const Coef<CT>& c, const CT* QL, const CT* AL, int iL,
                                            const CT* QR, const CT* AR, int iR, const CT* gt1,
                                            const CT* gt2, CT pk[7]) {
  CT s[3], fb4;
  face_s<D>(c, QL, AL, iL, QR, AR, iR, s, fb4);
  face_packet_s<D>(c, s, fb4, QL, iL, QR, iR, gt1, gt2, pk);
}

// In-plane face values of one plane slot, each face once: s-vector and Fb[4] of the
// x-faces between shared columns fx and fx+1 (fx in [0, SX-2]) of every shared row, and
// of the y-faces between shared rows fy and fy+1 (fy in [0, SY-2]) of every shared
// column.  Layout F[4][NF]: x-face (row, fx) at row*(SX-1) + fx, y-face (fy, col) at
// NXF + fy*SX + col; component 3 is Fb[4].  The per-cell sums S_d of the file comment
// are two reads of these.
constexpr int NXF = SY * (SX - 1);
constexpr int NYF = (SY - 1) * SX;
constexpr int NF = NXF + NYF;

template <class CT>
__device__ __forceinline__ const CT& xf(const CT* F, int j, int row, int fx) {
  return F[j * NF + row * (SX - 1) + fx];
}
template <class CT>
__device__ __forceinline__ const CT& yf(const CT* F, int j, int fy, int col) {
  return F[j * NF + NXF + fy * SX + col];
}

// Face values of one plane slot, each face once.  Every thread computes its own cell's
// lower x-face (shared row ty+1, fx = tx) and lower y-face (fy = ty, column tx+1); the
// NRF remaining faces (x-faces of the halo rows and of the last column, y-faces of the
// last row and of the halo columns) go to threads t < NRF.
constexpr int NRF = NF - 2 * NT;
static_assert(NRF == 2 * (SX - 1) + TY + SX + 2 * TY, "remaining faces of a plane slot");

template <class CT>
__device__ __forceinline__ void store_face(CT* __restrict__ F, int t, const CT sv[3], CT fb4) {
#pragma unroll
  for (int j = 0; j < 3; ++j) F[j * NF + t] = sv[j];
  F[3 * NF + t] = fb4;
}

template <class CT>
__device__ __forceinline__ void fill_faces(CT* __restrict__ F, const CT* __restrict__ sQ,
                                           const CT* __restrict__ sA, const Coef<CT>& c, int slot) {
  const CT* Q = sQ + slot * 5 * SP;
  const CT* A = sA + slot * 5 * SP;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  CT sv[3], fb4;
  {
    const int iL = (ty + 1) * SX + tx;
    face_s<0>(c, Q, A, iL, Q, A, iL + 1, sv, fb4);
    store_face(F, (ty + 1) * (SX - 1) + tx, sv, fb4);
  }
  {
    const int iL = ty * SX + tx + 1;
    face_s<1>(c, Q, A, iL, Q, A, iL + SX, sv, fb4);
    store_face(F, NXF + iL, sv, fb4);
  }
  const int t = threadIdx.x;
  if (t < NRF) {
    if (t < 2 * (SX - 1) + TY) {
      // x-faces: halo row 0, halo row SY-1, then the last face (fx = SX-2) of rows 1..TY
      int row, fx;
      if (t < SX - 1) {
        row = 0;
        fx = t;
      } else if (t < 2 * (SX - 1)) {
        row = SY - 1;
        fx = t - (SX - 1);
      } else {
        row = 1 + t - 2 * (SX - 1);
        fx = SX - 2;
      }
      const int iL = row * SX + fx;
      face_s<0>(c, Q, A, iL, Q, A, iL + 1, sv, fb4);
      store_face(F, row * (SX - 1) + fx, sv, fb4);
    } else {
      // y-faces: the last row of faces (fy = TY) at every column, then columns 0 and SX-1
      const int r = t - (2 * (SX - 1) + TY);
      int fy, col;
      if (r < SX) {
        fy = TY;
        col = r;
      } else {
        fy = (r - SX) >> 1;
        col = ((r - SX) & 1) ? SX - 1 : 0;
      }
      const int iL = fy * SX + col;
      face_s<1>(c, Q, A, iL, Q, A, iL + SX, sv, fb4);
      store_face(F, NXF + iL, sv, fb4);
    }
  }
}

// S_x[2], S_y[2] and S_x[0] + S_y[1] of the thread's own cell (shared row ty+1, column
// tx+1): the only components of the neighbouring planes' sums the assembly uses.
template <class CT>
__device__ __forceinline__ void own_S(const CT* F, int ty, int tx, CT o[3]) {
  o[0] = xf(F, 2, ty + 1, tx) + xf(F, 2, ty + 1, tx + 1);
  o[1] = yf(F, 2, ty, tx + 1) + yf(F, 2, ty + 1, tx + 1);
  o[2] = (xf(F, 0, ty + 1, tx) + xf(F, 0, ty + 1, tx + 1)) + (yf(F, 1, ty, tx + 1) + yf(F, 1, ty + 1, tx + 1));
}

template <class CT>
__device__ __forceinline__ void xpacket(const CT* sQ, const CT* F0, const Coef<CT>& c, int sm,
                                        int s0, int sp, int row, int fx, CT pk[7]) {
  const int iL = row * SX + fx, iR = iL + 1;
  const CT* Q0 = sQ + s0 * 5 * SP;
  const CT* Qm = sQ + sm * 5 * SP;
  const CT* Qp = sQ + sp * 5 * SP;
  // the four tangential derivatives the stress row reads: u_x along y and z, u_y along
  // y, u_z along z
  CT gy[3] = {CT(0), CT(0), CT(0)}, gz[3] = {CT(0), CT(0), CT(0)};
  {
    const CT* u0 = Q0 + SP;
    diff4_pair(u0[iL + SX], u0[iL - SX], u0[iR + SX], u0[iR - SX], c.i4dx[1], Qp[SP + iL], Qm[SP + iL],
               Qp[SP + iR], Qm[SP + iR], c.i4dx[2], gy[0], gz[0]);
    const CT* v0 = Q0 + 2 * SP;
    diff4_pair(v0[iL + SX], v0[iL - SX], v0[iR + SX], v0[iR - SX], c.i4dx[1], Qp[3 * SP + iL],
               Qm[3 * SP + iL], Qp[3 * SP + iR], Qm[3 * SP + iR], c.i4dx[2], gy[1], gz[2]);
  }
  const CT sv[3] = {xf(F0, 0, row, fx), xf(F0, 1, row, fx), xf(F0, 2, row, fx)};
  face_packet_s<0>(c, sv, xf(F0, 3, row, fx), Q0, iL, Q0, iR, gy, gz, pk);
}

template <class CT>
__device__ __forceinline__ void ypacket(const CT* sQ, const CT* F0, const Coef<CT>& c, int sm,
                                        int s0, int sp, int fy, int col, CT pk[7]) {
  const int iL = fy * SX + col, iR = iL + SX;
  const CT* Q0 = sQ + s0 * 5 * SP;
  const CT* Qm = sQ + sm * 5 * SP;
  const CT* Qp = sQ + sp * 5 * SP;
  // the four tangential derivatives the stress row reads: u_y along z and x, u_z along
  // z, u_x along x
  CT gz[3] = {CT(0), CT(0), CT(0)}, gx[3] = {CT(0), CT(0), CT(0)};
  {
    const CT* v0 = Q0 + 2 * SP;
    diff4_pair(Qp[2 * SP + iL], Qm[2 * SP + iL], Qp[2 * SP + iR], Qm[2 * SP + iR], c.i4dx[2], v0[iL + 1],
               v0[iL - 1], v0[iR + 1], v0[iR - 1], c.i4dx[0], gz[1], gx[1]);
    const CT* u0 = Q0 + SP;
    diff4_pair(Qp[3 * SP + iL], Qm[3 * SP + iL], Qp[3 * SP + iR], Qm[3 * SP + iR], c.i4dx[2], u0[iL + 1],
               u0[iL - 1], u0[iR + 1], u0[iR - 1], c.i4dx[0], gz[2], gx[0]);
  }
  const CT sv[3] = {yf(F0, 0, fy, col), yf(F0, 1, fy, col), yf(F0, 2, fy, col)};
  face_packet_s<1>(c, sv, yf(F0, 3, fy, col), Q0, iL, Q0, iR, gz, gx, pk);
}

template <class CT>
__device__ __forceinline__ void zpacket(const CT* sQ, const Coef<CT>& c, int sL, int sR, int i,
                                        const CT s[3], CT fb4, CT pk[7]) {
  const CT* QL = sQ + sL * 5 * SP;
  const CT* QR = sQ + sR * 5 * SP;
  // the four tangential derivatives the stress row reads: u_z along x and y, u_x along
  // x, u_y along y
  CT gx[3] = {CT(0), CT(0), CT(0)}, gy[3] = {CT(0), CT(0), CT(0)};
  {
    const CT* a = QL + 3 * SP;
    const CT* bq = QR + 3 * SP;
    diff4_pair(a[i + 1], a[i - 1], bq[i + 1], bq[i - 1], c.i4dx[0], a[i + SX], a[i - SX], bq[i + SX],
               bq[i - SX], c.i4dx[1], gx[2], gy[2]);
    const CT* ua = QL + SP;
    const CT* ub = QR + SP;
    const CT* va = QL + 2 * SP;
    const CT* vb = QR + 2 * SP;
    diff4_pair(ua[i + 1], ua[i - 1], ub[i + 1], ub[i - 1], c.i4dx[0], va[i + SX], va[i - SX], vb[i + SX],
               vb[i - SX], c.i4dx[1], gx[0], gy[1]);
  }
  face_packet_s<2>(c, s, fb4, QL, i, QR, i, gx, gy, pk);
}

// Roe part of a face packet: the adjoints of the two cells' primitives from the Roe
// dissipation, pk[0..4] for the left cell and pk[5..9] for the right cell, for the
// face adjoint Db = (a_L - a_R) / dx_D (D enters the face flux with the sign of F^v).
template <int D, class CT>
__device__ __forceinline__ void roe_packet(const Coef<CT>& c, const CT* QL, const CT* AL, int iL,
                                           const CT* QR, const CT* AR, int iR, CT* pk) {
  CT qL[5], qR[5], Db[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = QL[v * SP + iL];
    qR[v] = QR[v * SP + iR];
    Db[v] = (AL[v * SP + iL] - AR[v * SP + iR]) * c.idx[D];
  }
  roe_dissipation_adj<D>(c, qL, qR, Db, pk, pk + 5);
}

// z-face s-vectors between plane slots sL and sR at every shared column: the thread's own
// column ic (its s-vector and Fb[4] also returned for its z-packet) and the NH halo
// positions of the slot (rows 0 and SY-1, then columns 0 and SX-1 of rows 1..TY) by
// threads t < NH.
constexpr int NH = 2 * SX + 2 * TY;
static_assert(NH + NT == SP, "halo positions of a plane slot");

template <class CT>
__device__ __forceinline__ void fill_Z(CT* __restrict__ Z, const CT* __restrict__ sQ,
                                       const CT* __restrict__ sA, const Coef<CT>& c, int sL, int sR, int ic,
                                       CT s_own[3], CT& fb_own) {
  const CT* QL = sQ + sL * 5 * SP;
  const CT* AL = sA + sL * 5 * SP;
  const CT* QR = sQ + sR * 5 * SP;
  const CT* AR = sA + sR * 5 * SP;
  face_s<2>(c, QL, AL, ic, QR, AR, ic, s_own, fb_own);
#pragma unroll
  for (int j = 0; j < 3; ++j) Z[j * SP + ic] = s_own[j];
  const int t = threadIdx.x;
  if (t < NH) {
    int i;
    if (t < SX) i = t;
    else if (t < 2 * SX) i = (SY - 1) * SX + (t - SX);
    else {
      const int r = t - 2 * SX;
      i = (1 + (r >> 1)) * SX + ((r & 1) ? SX - 1 : 0);
    }
    CT sv[3], f;
    face_s<2>(c, QL, AL, i, QR, AR, i, sv, f);
#pragma unroll
    for (int j = 0; j < 3; ++j) Z[j * SP + i] = sv[j];
  }
}

}  // namespace

// Resident CTAs per SM the register allocation is held to (for the 32 x 4 tile; half
// as many CTAs of twice the threads for the 32 x 8 tile): 4 for FP32 (the shared memory
// allows 4), 3 for FP32 with Roe dissipation, 2 for FP64.
template <class CT, bool ROE> struct AdjMinBlocks { static constexpr int value = NT >= 256 ? 1 : 2; };
template <> struct AdjMinBlocks<float, false> { static constexpr int value = 512 / NT; };
template <> struct AdjMinBlocks<float, true> { static constexpr int value = NT >= 256 ? 1 : 3; };

// values per face packet: 7 (viscous and face velocity), plus 10 with Roe dissipation
template <bool ROE> constexpr int npk() { return ROE ? 17 : 7; }

template <class CT, class TIN, class TA, class TST, bool ROE>
__global__ void __launch_bounds__(NT, AdjMinBlocks<CT, ROE>::value) k_adj_stage(GridDesc g, Coef<CT> c, AdjArgs<TIN, TA, TST> a) {
  pdl_enter();
  constexpr int NPK = npk<ROE>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* sQ = reinterpret_cast<CT*>(smem_raw);   // [3][5][SP] primal primitives
  CT* sA = sQ + 3 * 5 * SP;                    // [3][5][SP] adjoint input a
  CT* sF = sA + 3 * 5 * SP;                    // [2][4][NF] in-plane face s-vectors, Fb[4]
  CT* sZ = sF + 2 * 4 * NF;                    // [2][3][SP] z-face s-vectors
  CT* sFX = sZ + 2 * 3 * SP;                   // [NPK][TY][TX+1]
  CT* sFY = sFX + NPK * TY * (TX + 1);         // [NPK][TY+1][TX]
  CT* sN = sFY + NPK * (TY + 1) * TX;          // [3][SP] added viscosity nu (when given)
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  int b, x0, y0, kz0, kz1;
  march_range<TX, TY>(g, b, x0, y0, kz0, kz1);
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < g.nx && gy < g.ny;
  const int cp = valid ? gy * g.nx + gx : 0;   // the thread's cell within a plane
  const size_t boxoff = (size_t)b * 5 * g.cells;
  const AdjHalo hal = adj_halo(g, x0, y0);
  const bool with_nu = a.nu != nullptr || a.nud != nullptr;
  auto slot = [&](int k) { return (k - kz0 + 1) % 3; };
  auto zslot = [&](int k) { return (k - kz0 + 1) & 1; };   // z-face k + 1/2
  auto fslot = [&](int k) { return sF + ((k - kz0 + 1) & 1) * 4 * NF; };   // faces of plane k

  {
    AdjPlaneRegs<CT> p0, p1, p2;
    adj_plane_load(p0, g, boxoff, b, kz0 - 1, hal, a.W, a.A, a.ca, a.nu, a.nud);
    adj_plane_load(p1, g, boxoff, b, kz0, hal, a.W, a.A, a.ca, a.nu, a.nud);
    adj_plane_load(p2, g, boxoff, b, kz0 + 1, hal, a.W, a.A, a.ca, a.nu, a.nud);
    adj_plane_store(p0, sQ + slot(kz0 - 1) * 5 * SP, sA + slot(kz0 - 1) * 5 * SP, sN + slot(kz0 - 1) * SP,
                    with_nu);
    adj_plane_store(p1, sQ + slot(kz0) * 5 * SP, sA + slot(kz0) * 5 * SP, sN + slot(kz0) * SP, with_nu);
    adj_plane_store(p2, sQ + slot(kz0 + 1) * 5 * SP, sA + slot(kz0 + 1) * 5 * SP, sN + slot(kz0 + 1) * SP,
                    with_nu);
  }
  __syncthreads();
  fill_faces(fslot(kz0 - 1), sQ, sA, c, slot(kz0 - 1));
  fill_faces(fslot(kz0), sQ, sA, c, slot(kz0));
  const int ic = (ty + 1) * SX + (tx + 1);
  CT zs[3], zf;
  fill_Z(sZ + zslot(kz0 - 1) * 3 * SP, sQ, sA, c, slot(kz0 - 1), slot(kz0), ic, zs, zf);
  CT zlo[NPK], zhi[NPK];
  zpacket(sQ, c, slot(kz0 - 1), slot(kz0), ic, zs, zf, zlo);
  if constexpr (ROE)
    roe_packet<2>(c, sQ + slot(kz0 - 1) * 5 * SP, sA + slot(kz0 - 1) * 5 * SP, ic, sQ + slot(kz0) * 5 * SP,
                  sA + slot(kz0) * 5 * SP, ic, zlo + 7);
  __syncthreads();
  // own-cell S sums of planes k-1 and k, carried in registers along the march
  CT own_m[3], own_0[3];
  own_S(fslot(kz0 - 1), ty, tx, own_m);
  own_S(fslot(kz0), ty, tx, own_0);
  __syncthreads();

  for (int k = kz0; k < kz1; ++k) {
    const int sm = slot(k - 1), s0 = slot(k), sp = slot(k + 1);
    const bool more = k + 1 < kz1;
    AdjPlaneRegs<CT> pf;
    if (more) adj_plane_load(pf, g, boxoff, b, k + 2, hal, a.W, a.A, a.ca, a.nu, a.nud);
    // per-cell operands of the assembly and epilogue, loaded ahead of the face work
    const size_t pbase = boxoff + (size_t)k * g.plane;   // component 0 of plane k
    const size_t fc = (size_t)g.cells;
    const long long n5 = 5 * g.cells * g.batch;           // field extent (debug bounds checks)
    (void)n5;
    CT gin[5] = {CT(0), CT(0), CT(0), CT(0), CT(0)};
    CT lfv[5] = {CT(0), CT(0), CT(0), CT(0), CT(0)};
    if (valid) {
      if (a.Gin) {
#pragma unroll
        for (int v = 0; v < 5; ++v) gin[v] = NS_LD(g, a.Gin, pbase + v * fc, cp, n5);
      }
      if (a.Anext) {
#pragma unroll
        for (int v = 0; v < 5; ++v) lfv[v] = NS_LD(g, a.lamf, pbase + v * fc, cp, n5);
      }
    }
    const CT* F0 = fslot(k);
    fill_faces(fslot(k + 1), sQ, sA, c, sp);
    fill_Z(sZ + zslot(k) * 3 * SP, sQ, sA, c, s0, sp, ic, zs, zf);
    {
      const CT* Q0 = sQ + s0 * 5 * SP;
      const CT* A0 = sA + s0 * 5 * SP;
      CT pkx[NPK], pky[NPK];
      xpacket(sQ, F0, c, sm, s0, sp, ty + 1, tx, pkx);
      if constexpr (ROE) roe_packet<0>(c, Q0, A0, ic - 1, Q0, A0, ic, pkx + 7);
      ypacket(sQ, F0, c, sm, s0, sp, ty, tx + 1, pky);
      if constexpr (ROE) roe_packet<1>(c, Q0, A0, ic - SX, Q0, A0, ic, pky + 7);
      zpacket(sQ, c, s0, sp, ic, zs, zf, zhi);
      if constexpr (ROE)
        roe_packet<2>(c, Q0, A0, ic, sQ + sp * 5 * SP, sA + sp * 5 * SP, ic, zhi + 7);
#pragma unroll
      for (int v = 0; v < NPK; ++v) sFX[(v * TY + ty) * (TX + 1) + tx] = pkx[v];
#pragma unroll
      for (int v = 0; v < NPK; ++v) sFY[(v * (TY + 1) + ty) * TX + tx] = pky[v];
    }
    if (tid < TX) {
      CT pk[NPK];
      ypacket(sQ, F0, c, sm, s0, sp, TY, tid + 1, pk);
      if constexpr (ROE) {
        const int iL = TY * SX + tid + 1;
        roe_packet<1>(c, sQ + s0 * 5 * SP, sA + s0 * 5 * SP, iL, sQ + s0 * 5 * SP, sA + s0 * 5 * SP, iL + SX,
                      pk + 7);
      }
#pragma unroll
      for (int v = 0; v < NPK; ++v) sFY[(v * (TY + 1) + TY) * TX + tid] = pk[v];
    } else if (tid < TX + TY) {
      CT pk[NPK];
      const int r = tid - TX;
      xpacket(sQ, F0, c, sm, s0, sp, r + 1, TX, pk);
      if constexpr (ROE) {
        const int iL = (r + 1) * SX + TX;
        roe_packet<0>(c, sQ + s0 * 5 * SP, sA + s0 * 5 * SP, iL, sQ + s0 * 5 * SP, sA + s0 * 5 * SP, iL + 1,
                      pk + 7);
      }
#pragma unroll
      for (int v = 0; v < NPK; ++v) sFX[(v * TY + r) * (TX + 1) + TX] = pk[v];
    }
    // the assembly reads plane k-1 only at the own cell: keep those values so that plane
    // k+2 can replace plane k-1 in the ring right after the barrier
    CT am[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) am[v] = sA[(sm * 5 + v) * SP + ic];
    const CT nzm = with_nu ? sN[sm * SP + ic] : CT(0);
    __syncthreads();
    if (more) adj_plane_store(pf, sQ + slot(k + 2) * 5 * SP, sA + slot(k + 2) * 5 * SP, sN + slot(k + 2) * SP,
                              with_nu);

    CT own_p[3] = {CT(0), CT(0), CT(0)};
    if (valid) {
      const CT* Q0 = sQ + s0 * 5 * SP;
      const CT* A0 = sA + s0 * 5 * SP;
      const CT* Ap = sA + sp * 5 * SP;
      const CT* Zl = sZ + zslot(k - 1) * 3 * SP;
      const CT* Zh = sZ + zslot(k) * 3 * SP;
      // ---- viscous: primitive adjoints of (u1, u2, u3, e)
      CT qb[4];
      const CT h = CT(0.5);
      {
        const int fl = ty * (TX + 1) + tx;
        const int yl = ty * TX + tx;
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const CT xl = sFX[v * TY * (TX + 1) + fl], xh = sFX[v * TY * (TX + 1) + fl + 1];
          const CT yl_ = sFY[v * (TY + 1) * TX + yl], yh = sFY[v * (TY + 1) * TX + yl + TX];
          const CT uxl = sFX[(4 + v) * TY * (TX + 1) + fl], uxh = sFX[(4 + v) * TY * (TX + 1) + fl + 1];
          const CT uyl = sFY[(4 + v) * (TY + 1) * TX + yl], uyh = sFY[(4 + v) * (TY + 1) * TX + yl + TX];
          qb[v] = (xl - xh) * c.idx[0] + (yl_ - yh) * c.idx[1] + (zlo[v] - zhi[v]) * c.idx[2] +
                  h * (uxl + uxh + uyl + uyh + zlo[4 + v] + zhi[4 + v]);
        }
        qb[3] = (sFX[3 * TY * (TX + 1) + fl] - sFX[3 * TY * (TX + 1) + fl + 1]) * c.idx[0] +
                (sFY[3 * (TY + 1) * TX + yl] - sFY[3 * (TY + 1) * TX + yl + TX]) * c.idx[1] +
                (zlo[3] - zhi[3]) * c.idx[2];
      }
      {
        // tangential parts, T[k][l] differenced along l
        const CT m = c.mu, m23 = CT(-2.0 / 3.0) * c.mu;
        const int il = ic - 1, ir = ic + 1, idn = ic - SX, iup = ic + SX;
        // S_z at a plane-k position = Zl + Zh
        auto Sz = [&](int j, int i) { return Zl[j * SP + i] + Zh[j * SP + i]; };
        // l = x (neighbours ic -+ 1): T[y][x] = mu S_y[x], T[z][x] = mu S_z[x],
        //                            T[x][x] = -2/3 mu (S_y[y] + S_z[z])
        // S_y[j] at il = (ty+1, tx) and ir = (ty+1, tx+2); S_x[j] at idn = (ty, tx+1) and
        // iup = (ty+2, tx+1): sums of the two in-plane faces of each cell (plane k)
        auto Syl = [&](int j) { return yf(F0, j, ty, tx) + yf(F0, j, ty + 1, tx); };
        auto Syr = [&](int j) { return yf(F0, j, ty, tx + 2) + yf(F0, j, ty + 1, tx + 2); };
        auto Sxd = [&](int j) { return xf(F0, j, ty, tx) + xf(F0, j, ty, tx + 1); };
        auto Sxu = [&](int j) { return xf(F0, j, ty + 2, tx) + xf(F0, j, ty + 2, tx + 1); };
        qb[0] = qb[0] + m23 * ((Syl(1) + Sz(2, il)) - (Syr(1) + Sz(2, ir))) * c.i4dx[0];
        qb[1] = qb[1] + m * (Syl(0) - Syr(0)) * c.i4dx[0];
        qb[2] = qb[2] + m * (Sz(0, il) - Sz(0, ir)) * c.i4dx[0];
        // l = y (neighbours ic -+ SX): T[x][y] = mu S_x[y], T[z][y] = mu S_z[y],
        //                             T[y][y] = -2/3 mu (S_x[x] + S_z[z])
        qb[0] = qb[0] + m * (Sxd(1) - Sxu(1)) * c.i4dx[1];
        qb[1] = qb[1] + m23 * ((Sxd(0) + Sz(2, idn)) - (Sxu(0) + Sz(2, iup))) * c.i4dx[1];
        qb[2] = qb[2] + m * (Sz(1, idn) - Sz(1, iup)) * c.i4dx[1];
        // l = z (planes k -+ 1): T[x][z] = mu S_x[z], T[y][z] = mu S_y[z],
        //                       T[z][z] = -2/3 mu (S_x[x] + S_y[y])
        own_S(fslot(k + 1), ty, tx, own_p);
        qb[0] = qb[0] + m * (own_m[0] - own_p[0]) * c.i4dx[2];
        qb[1] = qb[1] + m * (own_m[1] - own_p[1]) * c.i4dx[2];
        qb[2] = qb[2] + m23 * (own_m[2] - own_p[2]) * c.i4dx[2];
      }
      // ---- convective part and pull-back to conservative variables
      const CT rho = Q0[ic];
      const CT u[3] = {Q0[SP + ic], Q0[2 * SP + ic], Q0[3 * SP + ic]};
      const CT e = Q0[4 * SP + ic];
      const CT ir_ = CT(1) / rho;
      const CT Esp = e + h * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);   // rho E / rho
      const CT p = c.gm1 * rho * e;
      const CT rE = rho * Esp;
      CT rb = CT(0), mb[3] = {CT(0), CT(0), CT(0)}, Eb = CT(0), pb = CT(0);
      CT ub[3] = {qb[0], qb[1], qb[2]};
      CT eb = qb[3];
      if constexpr (ROE) {
        // Roe dissipation: the right-cell part of the lower faces and the left-cell part
        // of the upper faces, as adjoints of (rho, u, e)
        const int fl = ty * (TX + 1) + tx;
        const int yl = ty * TX + tx;
        CT rs[5];
#pragma unroll
        for (int v = 0; v < 5; ++v)
          rs[v] = sFX[(12 + v) * TY * (TX + 1) + fl] + sFX[(7 + v) * TY * (TX + 1) + fl + 1] +
                  sFY[(12 + v) * (TY + 1) * TX + yl] + sFY[(7 + v) * (TY + 1) * TX + yl + TX] +
                  zlo[12 + v] + zhi[7 + v];
        rb = rs[0];
#pragma unroll
        for (int j = 0; j < 3; ++j) ub[j] = ub[j] + rs[1 + j];
        eb = eb + rs[4];
      }
      const int nb_lo[3] = {ic - 1, ic - SX, ic};
      const int nb_hi[3] = {ic + 1, ic + SX, ic};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const CT* Ahi = d == 2 ? Ap : A0;
        CT F[5];
#pragma unroll
        for (int v = 0; v < 5; ++v)
          F[v] = (Ahi[v * SP + nb_hi[d]] - (d == 2 ? am[v] : A0[v * SP + nb_lo[d]])) * c.hidx[d];
        const CT md = rho * u[d];
        mb[d] = mb[d] + F[0] + F[1] * u[0] + F[2] * u[1] + F[3] * u[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) ub[j] = ub[j] + F[1 + j] * md;
        pb = pb + F[1 + d] + F[4] * u[d];
        Eb = Eb + F[4] * u[d];
        ub[d] = ub[d] + F[4] * (rE + p);
      }
      rb = rb + c.gm1 * e * pb;
      eb = eb + c.gm1 * rho * pb;
      Eb = Eb + eb * ir_;
      rb = rb - eb * Esp * ir_;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        ub[j] = ub[j] - eb * u[j];
        mb[j] = mb[j] + ub[j] * ir_;
        rb = rb - ub[j] * u[j] * ir_;
      }
      CT gout[5] = {rb, mb[0], mb[1], mb[2], Eb};
      // ---- added adjoint viscosity L_nu a, times the factor of the component's state
      // variable (rho, rho u, rho E)
      if (with_nu) {
        const CT* N0 = sN + s0 * SP;
        const CT nc = N0[ic], nxm = N0[ic - 1], nxp = N0[ic + 1], nym = N0[ic - SX], nyp = N0[ic + SX],
                 nzp = sN[sp * SP + ic];
        const CT ix2 = c.idx[0] * c.idx[0], iy2 = c.idx[1] * c.idx[1], iz2 = c.idx[2] * c.idx[2];
        int v0 = 0;
        if constexpr (std::is_same<CT, float>::value) {
          // components (0, 1) and (2, 3) side by side in paired FP32 instructions
          const float2 fxp = f2(h * (nc + nxp), h * (nc + nxp)), fxm = f2(-h * (nc + nxm), -h * (nc + nxm));
          const float2 fyp = f2(h * (nc + nyp), h * (nc + nyp)), fym = f2(-h * (nc + nym), -h * (nc + nym));
          const float2 fzp = f2(h * (nc + nzp), h * (nc + nzp)), fzm = f2(-h * (nc + nzm), -h * (nc + nzm));
#pragma unroll
          for (int v = 0; v < 4; v += 2) {
            const float* Av = A0 + v * SP;
            const float* Aw = Av + SP;
            const float2 ac = f2(Av[ic], Aw[ic]);
            const float2 tx = __ffma2_rn(fxp, sub2(f2(Av[ic + 1], Aw[ic + 1]), ac),
                                         __fmul2_rn(fxm, sub2(ac, f2(Av[ic - 1], Aw[ic - 1]))));
            const float2 ty = __ffma2_rn(fyp, sub2(f2(Av[ic + SX], Aw[ic + SX]), ac),
                                         __fmul2_rn(fym, sub2(ac, f2(Av[ic - SX], Aw[ic - SX]))));
            const float2 tz = __ffma2_rn(fzp, sub2(f2(Ap[v * SP + ic], Ap[(v + 1) * SP + ic]), ac),
                                         __fmul2_rn(fzm, sub2(ac, f2(am[v], am[v + 1]))));
            const float2 L = __ffma2_rn(tz, f2(iz2, iz2), __ffma2_rn(ty, f2(iy2, iy2), __fmul2_rn(tx, f2(ix2, ix2))));
            const float2 gv = __ffma2_rn(f2(float(a.nus[v == 0 ? 0 : 1]), float(a.nus[1])), L, f2(gout[v], gout[v + 1]));
            gout[v] = gv.x;
            gout[v + 1] = gv.y;
          }
          v0 = 4;
        }
#pragma unroll
        for (int v = v0; v < 5; ++v) {
          const CT* Av = A0 + v * SP;
          const CT ac = Av[ic];
          CT L = (h * (nc + nxp) * (Av[ic + 1] - ac) - h * (nc + nxm) * (ac - Av[ic - 1])) * ix2 +
                 (h * (nc + nyp) * (Av[ic + SX] - ac) - h * (nc + nym) * (ac - Av[ic - SX])) * iy2 +
                 (h * (nc + nzp) * (Ap[v * SP + ic] - ac) - h * (nc + nzm) * (ac - am[v])) * iz2;
          gout[v] = gout[v] + CT(a.nus[v == 0 ? 0 : (v == 4 ? 2 : 1)]) * L;
        }
      }
      // ---- epilogue (each optional operand tested once per plane)
      CT gs[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) gs[v] = gin[v] + gout[v];
      if (a.Gout) {
#pragma unroll
        for (int v = 0; v < 5; ++v) NS_ST(g, a.Gout, pbase + v * fc, cp, n5, gs[v]);
      }
      if (a.lam_out) {
        double lv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) lv[v] = widen(gs[v]);
        if (a.lam_in) {
#pragma unroll
          for (int v = 0; v < 5; ++v) lv[v] = NS_LD(g, a.lam_in, pbase + v * fc, cp, n5) + lv[v];
        }
        if (a.obj_ndsc && (gx == a.obj_iL || gx == a.obj_iR)) {
          // the objective source of this step on the plane's two columns, added after
          // the stage products (the order of the separate scatter it replaces)
          const int nf = g.ny * g.nz;
          const double* Af = a.obj_aface + ((size_t)b * nf + (size_t)k * g.ny + gy) * 5;
          const double NoD = a.obj_ndsc[2 * b], sc = a.obj_ndsc[2 * b + 1];
          const int reps = (gx == a.obj_iL ? 1 : 0) + (gx == a.obj_iR ? 1 : 0);
          for (int q = 0; q < reps; ++q) {
#pragma unroll
            for (int v = 0; v < 5; ++v) lv[v] += sc * (Af[v] - (v == 0 ? NoD : 0.0));
          }
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) NS_ST(g, a.lam_out, pbase + v * fc, cp, n5, lv[v]);
        if (a.lam_out_mirror) {
#pragma unroll
          for (int v = 0; v < 5; ++v) NS_ST(g, a.lam_out_mirror, pbase + v * fc, cp, n5, cvt<TST>(lv[v]));
        }
      }
      if (a.Anext) {
#pragma unroll
        for (int v = 0; v < 5; ++v)
          NS_ST(g, a.Anext, pbase + v * fc, cp, n5, CT(a.cl) * lfv[v] + CT(a.cg) * gout[v] + CT(a.cs) * gs[v]);
      }
      if (a.SBout || a.sbar) {
        CT ss[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) ss[v] = A0[v * SP + ic];
        if (a.SBin) {
#pragma unroll
          for (int v = 0; v < 5; ++v) ss[v] = NS_LD(g, a.SBin, pbase + v * fc, cp, n5) + ss[v];
        }
        if (a.SBout) {
#pragma unroll
          for (int v = 0; v < 5; ++v) NS_ST(g, a.SBout, pbase + v * fc, cp, n5, ss[v]);
        }
        if (a.sbar) {
#pragma unroll
          for (int v = 0; v < 5; ++v) NS_ST(g, a.sbar, pbase + v * fc, cp, n5, NS_LD(g, a.sbar, pbase + v * fc, cp, n5) + widen(ss[v]));
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NPK; ++v) zlo[v] = zhi[v];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      own_m[j] = own_0[j];
      own_0[j] = own_p[j];
    }
    __syncthreads();   // plane k+2 visible; packets, faces and z-faces free
  }
}

template <class CT, bool ROE>
size_t adj_smem_bytes() {
  constexpr int NPK = npk<ROE>();
  return sizeof(CT) *
         (3 * 5 * SP * 2 + 2 * 4 * NF + 2 * 3 * SP + NPK * TY * (TX + 1) + NPK * (TY + 1) * TX + 3 * SP);
}

template <class CT, class TIN, class TA, class TST, bool ROE>
static cudaError_t launch_adj_variant(const GridDesc& g, const Coef<CT>& c, const AdjArgs<TIN, TA, TST>& a,
                                     cudaStream_t st) {
  const size_t smem = adj_smem_bytes<CT, ROE>();
  auto kern = k_adj_stage<CT, TIN, TA, TST, ROE>;
  static MarchShape<TX, TY> shape;
  int ctas = 0;
  cudaError_t e = shape.get(kern, smem, g, "NS_ADJ_CTAS", ctas);
  if (e != cudaSuccess) return e;
  e = launch_pdl(kern, dim3(ctas), dim3(NT), smem, st, g, c, a);
  count_launch();
  return e;
}

}  // namespace adjk

template <class CT, class TIN, class TA, class TST>
cudaError_t launch_adj_stage(const GridDesc& g, const Coef<CT>& c, const AdjArgs<TIN, TA, TST>& a,
                             cudaStream_t st) {
  return c.roe ? adjk::launch_adj_variant<CT, TIN, TA, TST, true>(g, c, a, st)
               : adjk::launch_adj_variant<CT, TIN, TA, TST, false>(g, c, a, st);
}

template cudaError_t launch_adj_stage<double, double, double, double>(
    const GridDesc&, const Coef<double>&, const AdjArgs<double, double, double>&, cudaStream_t);
template cudaError_t launch_adj_stage<float, float, float, float>(
    const GridDesc&, const Coef<float>&, const AdjArgs<float, float, float>&, cudaStream_t);

}  // namespace ns
