// Primal residual and fused Runge-Kutta stage kernel (Eq. e:navier, Eq. e:vector).
//
// R(w)_c = -sum_d (Phi_d(c+1/2) - Phi_d(c-1/2)) / dx_d + s_c with the face flux
// Phi = (F_L + F_R)/2 - F^v(face).  F^v uses the compact normal difference and the
// mean of the two cell-centred central differences for the tangential derivatives of
// (u1, u2, u3, e); the face velocity is the two-cell mean; alpha = gamma mu / Pr.
//
// One CTA = TX x TY columns x a range of planes.  Per plane: every thread computes its
// cell's lower x-face and lower y-face and the z-face above it; 36 extra threads
// compute the tile's upper x/y boundary faces; the z-face below is carried in
// registers from the previous plane.  Each face flux is thus evaluated once per tile.
//
// Epilogue (fused Runge-Kutta update): the stage increments are summed in the stage type,
// dacc = sum_i b_i dt k_i, and only the final stage forms w^{n+1} = w^n + dacc in FP64,
// one FP64 add per component and step:
//   dacc = (dacc_init ? 0 : dacc) + cacc R,   Wout = base + cout R + cd dacc,
//   wout = wbase + widen(dacc + cacc R).
// The same template instantiated on ns::Dual gives the tangent (dR/dw) wd.
#include <type_traits>

#include "ns_common.cuh"
#include "ns_kernels.h"
#include "ns_roe.cuh"

namespace ns {
namespace rk {

// Tile of the primal stage kernel: 32 x 8 columns (256 threads), which halves the
// y-halo share of the plane loads and of the boundary faces against the 32 x 4 tile.
constexpr int TY = 8;
constexpr int NT = TX * TY;
constexpr int SY = TY + 2;
constexpr int SP = SX * SY;

// Field reads: element off of the field part that starts at element base (base: box,
// plane and component, common to the CTA; off: the thread's in-plane offset).
template <class CT, class TIN>
struct Loader {
  const TIN* W;
  const double* Wd;
  const GridDesc* g;
  __device__ __forceinline__ CT ld(size_t base, int off) const {
    return cvt<CT>(NS_LD(*g, W, base, off, 5 * g->cells * g->batch));
  }
};
template <>
struct Loader<Dual, double> {
  const double* W;
  const double* Wd;
  const GridDesc* g;
  __device__ __forceinline__ Dual ld(size_t base, int off) const {
    const long long n = 5 * g->cells * g->batch;
    return Dual(NS_LD(*g, W, base, off, n), NS_LD(*g, Wd, base, off, n));
  }
};

// In-plane offsets, periodic wrap resolved, of this thread's two shared positions
// t = tid and t = tid + NT (the same in every plane of the CTA's range).
struct HaloOff {
  int o[2];
};
__device__ __forceinline__ HaloOff halo_offsets(const GridDesc& g, int x0, int y0) {
  HaloOff h;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int t = threadIdx.x + it * NT;
    const int ly = t / SX;
    const int lx = t - ly * SX;
    h.o[it] = t < SP ? wrap(y0 + ly - 1, g.ny) * g.nx + wrap(x0 + lx - 1, g.nx) : 0;
  }
  return h;
}

// Two-phase plane load used to overlap the next plane's global loads with the
// current plane's face fluxes: plane_load issues the loads into registers,
// plane_store converts to primitives and writes the ring slot after a barrier.
static_assert(SP <= 2 * NT, "a plane must fit two load rounds");
template <class CT>
struct PlaneRegs {
  CT v[2][5];
};

template <class CT, class L>
__device__ __forceinline__ void plane_load(PlaneRegs<CT>& r, const GridDesc& g, size_t boxoff, int k,
                                           const HaloOff& h, const L& in) {
  const size_t pb = boxoff + (size_t)wrap(k, g.nz) * g.plane;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    if (threadIdx.x + it * NT < SP) {
#pragma unroll
      for (int v = 0; v < 5; ++v) r.v[it][v] = in.ld(pb + v * (size_t)g.cells, h.o[it]);
    }
  }
}

template <class CT>
__device__ __forceinline__ void plane_store(const PlaneRegs<CT>& r, CT* __restrict__ sq) {
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int t = threadIdx.x + it * NT;
    if (t < SP) {
      const CT ir = one_over(r.v[it][0]);
      const CT u0 = r.v[it][1] * ir, u1 = r.v[it][2] * ir, u2 = r.v[it][3] * ir;
      sq[0 * SP + t] = r.v[it][0];
      sq[1 * SP + t] = u0;
      sq[2 * SP + t] = u1;
      sq[3 * SP + t] = u2;
      sq[4 * SP + t] = r.v[it][4] * ir - CT(0.5) * (u0 * u0 + u1 * u1 + u2 * u2);
    }
  }
}

// Face flux Phi_D between cells L and R given the tangential face gradients of
// (u1, u2, u3, e) along T1 = (D+1)%3 and T2 = (D+2)%3.  Only gt1[D], gt2[D] (the stress
// row's cross terms) and gt1[T1], gt2[T2] (the divergence) are read.
template <int D, bool ROE, class CT>
__device__ __forceinline__ void face_flux(const Coef<CT>& c, const CT* qL, const CT* qR,
                                          const CT* gt1, const CT* gt2, CT* phi) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  CT g[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    g[k][D] = (qR[1 + k] - qL[1 + k]) * c.idx[D];
    g[k][T1] = gt1[k];
    g[k][T2] = gt2[k];
  }
  const CT div = g[0][0] + g[1][1] + g[2][2];
  CT sig[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) sig[j] = c.mu * (g[j][D] + g[D][j]);
  sig[D] = sig[D] - CT(2.0 / 3.0) * c.mu * div;
  CT fv4 = c.alpha * g[3][D];
#pragma unroll
  for (int j = 0; j < 3; ++j) fv4 = fv4 + CT(0.5) * (qL[1 + j] + qR[1 + j]) * sig[j];
  if constexpr (std::is_same<CT, float>::value) {
    // the left and right cells' Euler fluxes side by side in paired FP32 instructions
    const float2 Q0 = f2(qL[0], qR[0]), Q4 = f2(qL[4], qR[4]), QD = f2(qL[1 + D], qR[1 + D]);
    const float2 P = __fmul2_rn(__fmul2_rn(f2(c.gm1, c.gm1), Q0), Q4);         // p
    const float2 M = __fmul2_rn(Q0, QD);                                          // rho u_D
    float2 K = __fmul2_rn(f2(qL[1], qR[1]), f2(qL[1], qR[1]));
    K = __ffma2_rn(f2(qL[2], qR[2]), f2(qL[2], qR[2]), K);
    K = __ffma2_rn(f2(qL[3], qR[3]), f2(qL[3], qR[3]), K);
    K = __fmul2_rn(f2(0.5f, 0.5f), K);                                          // |u|^2 / 2
    phi[0] = 0.5f * (M.x + M.y);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 T = __fmul2_rn(M, f2(qL[1 + k], qR[1 + k]));
      phi[1 + k] = 0.5f * (T.x + T.y) - sig[k];
    }
    phi[1 + D] = phi[1 + D] + 0.5f * (P.x + P.y);
    const float2 E = __ffma2_rn(P, QD, __fmul2_rn(M, __fadd2_rn(Q4, K)));
    phi[4] = 0.5f * (E.x + E.y) - fv4;
  } else {
    const CT pL = c.gm1 * qL[0] * qL[4];
    const CT pR = c.gm1 * qR[0] * qR[4];
    const CT mL = qL[0] * qL[1 + D];
    const CT mR = qR[0] * qR[1 + D];
    const CT kL = CT(0.5) * (qL[1] * qL[1] + qL[2] * qL[2] + qL[3] * qL[3]);
    const CT kR = CT(0.5) * (qR[1] * qR[1] + qR[2] * qR[2] + qR[3] * qR[3]);
    phi[0] = CT(0.5) * (mL + mR);
#pragma unroll
    for (int k = 0; k < 3; ++k) phi[1 + k] = CT(0.5) * (mL * qL[1 + k] + mR * qR[1 + k]) - sig[k];
    phi[1 + D] = phi[1 + D] + CT(0.5) * (pL + pR);
    phi[4] = CT(0.5) * (mL * (qL[4] + kL) + pL * qL[1 + D] + mR * (qR[4] + kR) + pR * qR[1 + D]) - fv4;
  }
  if constexpr (ROE) {
    CT Dv[5];
    roe_dissipation<D>(c, qL, qR, Dv);
#pragma unroll
    for (int v = 0; v < 5; ++v) phi[v] = phi[v] - Dv[v];
  }
}

template <class CT>
__device__ __forceinline__ const CT* qs(const CT* sQ, int slot, int v) {
  return sQ + (slot * 5 + v) * SP;
}

// x-face between shared cells (row, fx) and (row, fx+1); row/fx in shared coords.
template <bool ROE, class CT>
__device__ __forceinline__ void xface(const CT* sQ, const Coef<CT>& c, int sm, int s0, int sp,
                                      int row, int fx, CT* phi) {
  const int iL = row * SX + fx, iR = iL + 1;
  CT qL[5], qR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = qs(sQ, s0, v)[iL];
    qR[v] = qs(sQ, s0, v)[iR];
  }
  // the four tangential derivatives the flux reads: u_x along y and z, u_y along y, u_z
  // along z (face_flux)
  CT gy[4] = {CT(0), CT(0), CT(0), CT(0)}, gz[4] = {CT(0), CT(0), CT(0), CT(0)};
  {
    const CT* p0 = qs(sQ, s0, 1);
    diff4_pair(p0[iL + SX], p0[iL - SX], p0[iR + SX], p0[iR - SX], c.i4dx[1], qs(sQ, sp, 1)[iL],
               qs(sQ, sm, 1)[iL], qs(sQ, sp, 1)[iR], qs(sQ, sm, 1)[iR], c.i4dx[2], gy[0], gz[0]);
    const CT* v0 = qs(sQ, s0, 2);
    diff4_pair(v0[iL + SX], v0[iL - SX], v0[iR + SX], v0[iR - SX], c.i4dx[1], qs(sQ, sp, 3)[iL],
               qs(sQ, sm, 3)[iL], qs(sQ, sp, 3)[iR], qs(sQ, sm, 3)[iR], c.i4dx[2], gy[1], gz[2]);
  }
  face_flux<0, ROE>(c, qL, qR, gy, gz, phi);
}

// y-face between shared cells (fy, col) and (fy+1, col).
template <bool ROE, class CT>
__device__ __forceinline__ void yface(const CT* sQ, const Coef<CT>& c, int sm, int s0, int sp,
                                      int fy, int col, CT* phi) {
  const int iL = fy * SX + col, iR = iL + SX;
  CT qL[5], qR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = qs(sQ, s0, v)[iL];
    qR[v] = qs(sQ, s0, v)[iR];
  }
  // the four tangential derivatives the flux reads: u_y along z and x, u_z along z, u_x
  // along x
  CT gz[4] = {CT(0), CT(0), CT(0), CT(0)}, gx[4] = {CT(0), CT(0), CT(0), CT(0)};
  {
    const CT* v0 = qs(sQ, s0, 2);
    diff4_pair(qs(sQ, sp, 2)[iL], qs(sQ, sm, 2)[iL], qs(sQ, sp, 2)[iR], qs(sQ, sm, 2)[iR], c.i4dx[2],
               v0[iL + 1], v0[iL - 1], v0[iR + 1], v0[iR - 1], c.i4dx[0], gz[1], gx[1]);
    const CT* u0 = qs(sQ, s0, 1);
    diff4_pair(qs(sQ, sp, 3)[iL], qs(sQ, sm, 3)[iL], qs(sQ, sp, 3)[iR], qs(sQ, sm, 3)[iR], c.i4dx[2],
               u0[iL + 1], u0[iL - 1], u0[iR + 1], u0[iR - 1], c.i4dx[0], gz[2], gx[0]);
  }
  face_flux<1, ROE>(c, qL, qR, gz, gx, phi);
}

// z-face between slot sL (lower plane) and sR (upper plane) at shared cell index i.
template <bool ROE, class CT>
__device__ __forceinline__ void zface(const CT* sQ, const Coef<CT>& c, int sL, int sR, int i,
                                      CT* phi) {
  CT qL[5], qR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = qs(sQ, sL, v)[i];
    qR[v] = qs(sQ, sR, v)[i];
  }
  // the four tangential derivatives the flux reads: u_z along x and y, u_x along x, u_y
  // along y
  CT gx[4] = {CT(0), CT(0), CT(0), CT(0)}, gy[4] = {CT(0), CT(0), CT(0), CT(0)};
  {
    const CT* a = qs(sQ, sL, 3);
    const CT* bq = qs(sQ, sR, 3);
    diff4_pair(a[i + 1], a[i - 1], bq[i + 1], bq[i - 1], c.i4dx[0], a[i + SX], a[i - SX], bq[i + SX],
               bq[i - SX], c.i4dx[1], gx[2], gy[2]);
    const CT* ua = qs(sQ, sL, 1);
    const CT* ub = qs(sQ, sR, 1);
    const CT* va = qs(sQ, sL, 2);
    const CT* vb = qs(sQ, sR, 2);
    diff4_pair(ua[i + 1], ua[i - 1], ub[i + 1], ub[i - 1], c.i4dx[0], va[i + SX], va[i - SX], vb[i + SX],
               vb[i - SX], c.i4dx[1], gx[0], gy[1]);
  }
  face_flux<2, ROE>(c, qL, qR, gx, gy, phi);
}

// Resident CTAs per SM the register allocation is held to: 3 for FP32 (85 registers or
// fewer), 2 for FP32 with Roe dissipation, 1 for FP64 and the dual-number tangent.
template <class CT, bool ROE> struct RhsMinBlocks { static constexpr int value = 1; };
template <> struct RhsMinBlocks<float, false> { static constexpr int value = 3; };
template <> struct RhsMinBlocks<float, true> { static constexpr int value = 2; };

template <class CT, class TIN, class TST, bool ROE>
__global__ void __launch_bounds__(NT, RhsMinBlocks<CT, ROE>::value) k_rhs_stage(GridDesc g, Coef<CT> c, StageArgs<TIN, TST> a) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* sQ = reinterpret_cast<CT*>(smem_raw);          // [3][5][SP]
  CT* sFX = sQ + 3 * 5 * SP;                          // [5][TY][TX+1]
  CT* sFY = sFX + 5 * TY * (TX + 1);                  // [5][TY+1][TX]
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  Loader<CT, TIN> in{a.W, a.Wd, &g};
  int b, x0, y0, kz0, kz1;
  march_range<TX, TY>(g, b, x0, y0, kz0, kz1);
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < g.nx && gy < g.ny;
  const int cp = valid ? gy * g.nx + gx : 0;        // the thread's cell within a plane
  const size_t boxoff = (size_t)b * 5 * g.cells;
  const HaloOff h = halo_offsets(g, x0, y0);

  // ring slots: plane k-1, k, k+1 sit in slots (k-kz0) % 3, (k-kz0+1) % 3, (k-kz0+2) % 3
  {
    PlaneRegs<CT> p0, p1, p2;
    plane_load(p0, g, boxoff, kz0 - 1, h, in);
    plane_load(p1, g, boxoff, kz0, h, in);
    plane_load(p2, g, boxoff, kz0 + 1, h, in);
    plane_store(p0, sQ);
    plane_store(p1, sQ + 5 * SP);
    plane_store(p2, sQ + 2 * 5 * SP);
  }
  __syncthreads();
  const int ic = (ty + 1) * SX + (tx + 1);
  CT zlo[5], zhi[5];
  zface<ROE>(sQ, c, 0, 1, ic, zlo);

  // the march: at plane k the ring slots of planes k-1, k, k+1 are sm, s0, sp (sm = j
  // cycles 0, 1, 2).  A loop unrolled over the three rotations, with the slots as
  // compile-time constants, needs more registers than the 80 this kernel is held to and
  // measured slower.
  for (int k = kz0, j = 0; k < kz1; ++k, j = (j == 2 ? 0 : j + 1)) {
    const int sm = j, s0 = (sm + 1) % 3, sp = (sm + 2) % 3;
    const bool more = k + 1 < kz1;
    PlaneRegs<CT> pf;
    if (more) plane_load(pf, g, boxoff, k + 2, h, in);
    const size_t pb = boxoff + (size_t)k * g.plane;   // component 0 of plane k
    const long long n5 = 5 * g.cells * g.batch;        // field extent (debug bounds checks)
    (void)n5;
    // epilogue operands of this plane, issued before the face fluxes so that their
    // latency overlaps the flux arithmetic (scalar path)
    CT e_src[5], e_dacc[5], e_base[5];
    if constexpr (!std::is_same<CT, Dual>::value) {
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        e_src[v] = CT(0);
        e_dacc[v] = CT(0);
        e_base[v] = CT(0);
      }
      if (valid) {
        if (a.src) {
#pragma unroll
          for (int v = 0; v < 5; ++v) e_src[v] = cvt<CT>(NS_LD(g, a.src, pb + v * (size_t)g.cells, cp, n5));
        }
        if (a.dacc && !a.dacc_init) {
#pragma unroll
          for (int v = 0; v < 5; ++v) e_dacc[v] = CT(NS_LD(g, a.dacc, pb + v * (size_t)g.cells, cp, n5));
        }
        if (a.Wout) {
#pragma unroll
          for (int v = 0; v < 5; ++v) e_base[v] = CT(NS_LD(g, a.base, pb + v * (size_t)g.cells, cp, n5));
        }
      }
    }
    {
      CT phi[5];
      xface<ROE>(sQ, c, sm, s0, sp, ty + 1, tx, phi);
#pragma unroll
      for (int v = 0; v < 5; ++v) sFX[(v * TY + ty) * (TX + 1) + tx] = phi[v];
      yface<ROE>(sQ, c, sm, s0, sp, ty, tx + 1, phi);
#pragma unroll
      for (int v = 0; v < 5; ++v) sFY[(v * (TY + 1) + ty) * TX + tx] = phi[v];
    }
    zface<ROE>(sQ, c, s0, sp, ic, zhi);
    if (tid < TX) {
      CT phi[5];
      yface<ROE>(sQ, c, sm, s0, sp, TY, tid + 1, phi);
#pragma unroll
      for (int v = 0; v < 5; ++v) sFY[(v * (TY + 1) + TY) * TX + tid] = phi[v];
    } else if (tid < TX + TY) {
      CT phi[5];
      const int r = tid - TX;
      xface<ROE>(sQ, c, sm, s0, sp, r + 1, TX, phi);
#pragma unroll
      for (int v = 0; v < 5; ++v) sFX[(v * TY + r) * (TX + 1) + TX] = phi[v];
    }
    __syncthreads();
    // the epilogue reads only the face fluxes: plane k+2 replaces plane k-1 in the ring now
    if (more) plane_store(pf, sQ + sm * 5 * SP);
    if (valid) {
      CT R[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const CT fxp = sFX[(v * TY + ty) * (TX + 1) + tx + 1];
        const CT fxm = sFX[(v * TY + ty) * (TX + 1) + tx];
        const CT fyp = sFY[(v * (TY + 1) + ty + 1) * TX + tx];
        const CT fym = sFY[(v * (TY + 1) + ty) * TX + tx];
        R[v] = -((fxp - fxm) * c.idx[0] + (fyp - fym) * c.idx[1] + (zhi[v] - zlo[v]) * c.idx[2]);
      }
      if constexpr (std::is_same<CT, Dual>::value) {
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          const size_t o = pb + v * (size_t)g.cells + cp;
          if (!NS_IN_BOUNDS(g, o, n5)) continue;
          double Rv = R[v].v, Rd = R[v].d;
          if (a.src) Rv += a.src[o];
          if (a.srcd) Rd += a.srcd[o];
          const double iv = a.cacc * Rv, id = a.cacc * Rd;
          const double dv = (a.dacc && !a.dacc_init ? (double)a.dacc[o] : 0.0) + iv;
          const double dd = (a.daccd && !a.dacc_init ? a.daccd[o] : 0.0) + id;
          if (a.wout) a.wout[o] = (a.wbase ? a.wbase[o] : 0.0) + dv;
          else if (a.dacc) a.dacc[o] = dv;
          if (a.woutd) a.woutd[o] = (a.wbased ? a.wbased[o] : 0.0) + dd;
          else if (a.daccd) a.daccd[o] = dd;
          if (a.Wout) {
            a.Wout[o] = a.base[o] + a.cout * Rv + a.cd * dv;
            if (a.Woutd) a.Woutd[o] = a.based[o] + a.cout * Rd + a.cd * dd;
          }
        }
      } else {
        CT Rv[5], dv[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          Rv[v] = R[v] + e_src[v];
          const CT inc = CT(a.cacc) * Rv[v];
          dv[v] = e_dacc[v] + inc;
        }
        if (a.wout) {
          double e_wbase[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
          if (a.wbase) {
#pragma unroll
            for (int v = 0; v < 5; ++v) e_wbase[v] = NS_LD(g, a.wbase, pb + v * (size_t)g.cells, cp, n5);
          }
          if (a.wout_mirror) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const double wv = e_wbase[v] + widen(dv[v]);
              NS_ST(g, a.wout, pb + v * (size_t)g.cells, cp, n5, wv);
              NS_ST(g, a.wout_mirror, pb + v * (size_t)g.cells, cp, n5, cvt<TST>(wv));
            }
          } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) NS_ST(g, a.wout, pb + v * (size_t)g.cells, cp, n5, e_wbase[v] + widen(dv[v]));
          }
        } else if (a.dacc) {
#pragma unroll
          for (int v = 0; v < 5; ++v) NS_ST(g, a.dacc, pb + v * (size_t)g.cells, cp, n5, dv[v]);
        }
        if (a.Wout) {
#pragma unroll
          for (int v = 0; v < 5; ++v)
            NS_ST(g, a.Wout, pb + v * (size_t)g.cells, cp, n5, e_base[v] + CT(a.cout) * Rv[v] + CT(a.cd) * dv[v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) zlo[v] = zhi[v];
    __syncthreads();   // plane k+2 visible; face fluxes free
  }
}

}  // namespace rk

template <class CT>
size_t rhs_smem_bytes() {
  return sizeof(CT) * (3 * 5 * rk::SP + 5 * rk::TY * (TX + 1) + 5 * (rk::TY + 1) * TX);
}

template <class CT, class TIN, class TST, bool ROE>
static cudaError_t launch_rhs_variant(const GridDesc& g, const Coef<CT>& c, const StageArgs<TIN, TST>& a,
                                     cudaStream_t st) {
  const size_t smem = rhs_smem_bytes<CT>();
  auto kern = rk::k_rhs_stage<CT, TIN, TST, ROE>;
  static MarchShape<TX, rk::TY> shape;
  int ctas = 0;
  cudaError_t e = shape.get(kern, smem, g, "NS_RHS_CTAS", ctas);
  if (e != cudaSuccess) return e;
  e = launch_pdl(kern, dim3(ctas), dim3(rk::NT), smem, st, g, c, a);
  count_launch();
  return e;
}

template <class CT, class TIN, class TST>
cudaError_t launch_rhs_stage(const GridDesc& g, const Coef<CT>& c, const StageArgs<TIN, TST>& a,
                             cudaStream_t st) {
  return c.roe ? launch_rhs_variant<CT, TIN, TST, true>(g, c, a, st)
               : launch_rhs_variant<CT, TIN, TST, false>(g, c, a, st);
}

template cudaError_t launch_rhs_stage<double, double, double>(const GridDesc&, const Coef<double>&,
                                                              const StageArgs<double, double>&, cudaStream_t);
template cudaError_t launch_rhs_stage<float, float, float>(const GridDesc&, const Coef<float>&,
                                                           const StageArgs<float, float>&, cudaStream_t);
template cudaError_t launch_rhs_stage<Dual, double, double>(const GridDesc&, const Coef<Dual>&,
                                                            const StageArgs<double, double>&, cudaStream_t);

}  // namespace ns
