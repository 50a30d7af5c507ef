// Boundaries of a bounded box: characteristic (non-reflecting) inflow at x = 0 and
// outflow at x = L_x (section "Numerical methods"; the incoming characteristics are
// set there, section "Energy analysis"), and isothermal no-slip walls at y = 0 and
// y = L_y (the vane surface is isothermal, section "Problem setup"); z stays periodic.
//
// A bounded context works on the box padded by one ghost layer: ghost columns at
// x = -1 and x = nx (inflow, outflow), ghost rows at y = -1 and y = ny (walls), the
// rows built over the columns so that a corner is the wall's ghost of the inflow or
// outflow ghost.  The residual is the periodic residual of the padded box, cropped:
// the periodic stage kernels run unchanged on the padded box once its ghosts are
// filled (k_bc_ghosts).  The adjoint is the exact transpose of that map: the periodic
// transposed product runs on the padded box with a zero adjoint in the ghosts, and
// k_bc_adj_epilogue pulls each ghost's output back to the cell the ghost was built from
// through the transposed 5 x 5 ghost Jacobian (forward-mode dual numbers), rows first,
// then columns (the reverse of the padding's order).  The added adjoint viscosity
// passes no flux through the boundary faces, which keeps it symmetric and
// non-positive; the epilogue applies it on the unpadded box with those faces closed.
//
// Ghost states.  Inflow and outflow hold the boundary state of the x-direction Riemann
// invariants R+- = u1 +- 2c/(gamma-1): at the outflow R+, the entropy p/rho^gamma and
// the tangential velocity come from the adjacent cell and R- from the far field; at the
// inflow R- comes from the adjacent cell and the rest from the far field (subsonic flow
// along +x).  A wall ghost has the adjacent cell's density, its momentum reversed and
// the internal energy 2 e_w - e, so that the face velocity is zero and the face
// temperature is the wall's.
#include <cuda_runtime.h>

#include <type_traits>

#include "ns_common.cuh"
#include "ns_kernels.h"

namespace ns {

namespace {

__device__ __forceinline__ Dual dsqrt(Dual a) {
  const double r = sqrt(a.v);
  return Dual(r, 0.5 * a.d / r);
}
__device__ __forceinline__ Dual dpow(Dual a, double e) {
  const double r = pow(a.v, e);
  return Dual(r, e * pow(a.v, e - 1.0) * a.d);
}
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double dpow(double a, double e) { return pow(a, e); }
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ float dpow(float a, double e) { return powf(a, (float)e); }

// boundary state of a characteristic inflow (side 0) or outflow (side 1) ghost from the
// adjacent cell's conservative state wc
template <class T>
__device__ void char_state(const T wc[5], int side, const BcDesc& bc, T out[5]) {
  const double g = bc.gamma, k = 2.0 / (g - 1.0);
  const T rho = wc[0];
  const T u0 = wc[1] / rho, u1 = wc[2] / rho, u2 = wc[3] / rho;
  const T p = T(g - 1.0) * (wc[4] - T(0.5) * rho * (u0 * u0 + u1 * u1 + u2 * u2));
  const T c = dsqrt(T(g) * p / rho);
  const double rf = bc.far[0], uf1 = bc.far[1], uf2 = bc.far[2], uf3 = bc.far[3], pf = bc.far[4];
  const double cf = sqrt(g * pf / rf);
  T Rp, Rm, ent, ut2, ut3;
  if (side == 1) {
    Rp = u0 + T(k) * c;
    Rm = T(uf1 - k * cf);
    ent = p / dpow(rho, g);
    ut2 = u1;
    ut3 = u2;
  } else {
    Rp = T(uf1 + k * cf);
    Rm = u0 - T(k) * c;
    ent = T(pf / pow(rf, g));
    ut2 = T(uf2);
    ut3 = T(uf3);
  }
  const T ub = T(0.5) * (Rp + Rm);
  const T cb = T(0.25 * (g - 1.0)) * (Rp - Rm);
  const T rhob = dpow(cb * cb / (T(g) * ent), 1.0 / (g - 1.0));
  const T pb = rhob * cb * cb / T(g);
  out[0] = rhob;
  out[1] = rhob * ub;
  out[2] = rhob * ut2;
  out[3] = rhob * ut3;
  out[4] = pb / T(g - 1.0) + T(0.5) * rhob * (ub * ub + ut2 * ut2 + ut3 * ut3);
}

// isothermal no-slip wall ghost, bottom (side 0) or top (side 1)
template <class T>
__device__ void wall_state(const T wc[5], int side, const BcDesc& bc, T out[5]) {
  const T rho = wc[0];
  const T u0 = wc[1] / rho, u1 = wc[2] / rho, u2 = wc[3] / rho;
  const T k2 = T(0.5) * (u0 * u0 + u1 * u1 + u2 * u2);
  const T e = wc[4] / rho - k2;
  const T eg = T(2.0 * bc.wall_e[side]) - e;
  out[0] = rho;
  out[1] = -wc[1];
  out[2] = -wc[2];
  out[3] = -wc[3];
  out[4] = rho * (eg + k2);
}

struct Pad {
  int ix, iy;          // ghost widths in x and y (0 or 1)
  int nxp, nyp;        // padded sizes
  long long planep, cellsp;
};

__device__ __forceinline__ Pad pad_of(const GridDesc& g, const BcDesc& bc) {
  Pad p;
  p.ix = bc.inout;
  p.iy = bc.walls;
  p.nxp = g.nx + 2 * p.ix;
  p.nyp = g.ny + 2 * p.iy;
  p.planep = (long long)p.nxp * p.nyp;
  p.cellsp = p.planep * g.nz;
  return p;
}

// padded field (interior copied and converted, ghosts zero), ncomp components per box
template <class TO, class TI>
__global__ void k_bc_embed(GridDesc g, BcDesc bc, int ncomp, double scale, const TI* __restrict__ src,
                           TO* __restrict__ dst) {
  const Pad P = pad_of(g, bc);
  const long long n = P.cellsp * ncomp * g.batch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long bc_ = i / P.cellsp, r = i - bc_ * P.cellsp;
    const int z = (int)(r / P.planep);
    const long long rp = r - (long long)z * P.planep;
    const int yp = (int)(rp / P.nxp), xp = (int)(rp - (long long)yp * P.nxp);
    const int x = xp - P.ix, y = yp - P.iy;
    TO v = TO(0);
    if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
      const double s = (double)src[bc_ * g.cells + (long long)z * g.plane + (long long)y * g.nx + x];
      v = cvt<TO>(scale * s);
    }
    dst[i] = v;
  }
}

// interior of a padded field
template <class TO, class TI>
__global__ void k_bc_crop(GridDesc g, BcDesc bc, int ncomp, const TI* __restrict__ src, TO* __restrict__ dst) {
  const Pad P = pad_of(g, bc);
  const long long n = g.cells * ncomp * g.batch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long bc_ = i / g.cells, r = i - bc_ * g.cells;
    const int z = (int)(r / g.plane);
    const long long rr = r - (long long)z * g.plane;
    const int y = (int)(rr / g.nx), x = (int)(rr - (long long)y * g.nx);
    dst[i] = (TO)src[bc_ * P.cellsp + (long long)z * P.planep + (long long)(y + P.iy) * P.nxp + (x + P.ix)];
  }
}

template <class T>
__device__ __forceinline__ void load5(const T* f, long long o, long long stride, T v[5]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) v[k] = f[o + k * stride];
}

// the ghost layer of a padded state field, from its interior boundary cells
template <class T>
__global__ void k_bc_ghosts(GridDesc g, BcDesc bc, T* __restrict__ W) {
  const Pad P = pad_of(g, bc);
  // ghost cells per plane: the x columns' interior rows, then the y rows' full width
  const int nxg = P.ix ? 2 * g.ny : 0, nyg = P.iy ? 2 * P.nxp : 0;
  const long long per = (long long)(nxg + nyg) * g.nz;
  const long long n = per * g.batch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / per, r = i - b * per;
    const int z = (int)(r / (nxg + nyg));
    int j = (int)(r - (long long)z * (nxg + nyg));
    const long long box = b * 5 * P.cellsp + (long long)z * P.planep;
    auto at = [&](int xp, int yp) { return box + (long long)yp * P.nxp + xp; };
    T wc[5], gs[5];
    long long dst;
    if (j < nxg) {
      // inflow (side 0) or outflow (side 1) column at interior row y
      const int side = j / g.ny, y = j - side * g.ny;
      const int xc = side == 0 ? P.ix : P.ix + g.nx - 1;
      load5(W, at(xc, y + P.iy), P.cellsp, wc);
      char_state<T>(wc, side, bc, gs);
      dst = at(side == 0 ? 0 : P.nxp - 1, y + P.iy);
    } else {
      // wall rows over the full padded width; at a corner, the wall ghost of the
      // inflow or outflow ghost of the corner cell
      j -= nxg;
      const int side = j / P.nxp, xp = j - side * P.nxp;
      const int yc = side == 0 ? P.iy : P.iy + g.ny - 1;
      const int x = xp - P.ix;
      if (x >= 0 && x < g.nx) {
        load5(W, at(xp, yc), P.cellsp, wc);
      } else {
        T wi[5];
        load5(W, at(x < 0 ? P.ix : P.ix + g.nx - 1, yc), P.cellsp, wi);
        char_state<T>(wi, x < 0 ? 0 : 1, bc, wc);
      }
      wall_state<T>(wc, side, bc, gs);
      dst = at(xp, side == 0 ? 0 : P.nyp - 1);
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) W[dst + k * P.cellsp] = gs[k];
  }
}

// d = J^T h for the Jacobian J[i][k] = d ghost_i / d wc_k of a characteristic (kind 0)
// or wall (kind 1) ghost built from wc, by forward-mode dual numbers
__device__ void ghost_pullback(const double wc[5], int kind, int side, const BcDesc& bc, const double h[5],
                               double d[5]) {
#pragma unroll 1
  for (int k = 0; k < 5; ++k) {
    Dual x[5], o[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) x[m] = Dual(wc[m], m == k ? 1.0 : 0.0);
    if (kind == 0)
      char_state<Dual>(x, side, bc, o);
    else
      wall_state<Dual>(x, side, bc, o);
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < 5; ++i) acc += o[i].d * h[i];
    d[k] = acc;
  }
}

// The boundary epilogue of one transposed stage on a bounded box, per interior cell:
//   g   = gp(c) + the ghosts' outputs pulled back + L_nu a (boundary faces closed)
// then, as the periodic adjoint stage does:
//   mode 0 (transposed residual only):  out = g
//   mode 1 (a Runge-Kutta stage):        Gs = (first ? 0 : G) + g; G = Gs (not last);
//       a_next = cl lam + cg g + cs Gs (not last); lam_out = lam + Gs (last);
//       sbar += a (when sbar != null)
// gp: the transposed product on the padded box (FP64); W: the padded stage state
// (ghost inputs); A, sa: the stage's seed a = sa A (unpadded FP64).
template <class CT, class NU>
__global__ void k_bc_adj_epilogue(GridDesc g, BcDesc bc, const double* __restrict__ gp, const CT* __restrict__ W,
                                  const double* __restrict__ A, double sa, const NU* __restrict__ nu, double nus0,
                                  double nus1, double nus2, double i2x, double i2y, double i2z, int mode, int first,
                                  int last, const double* __restrict__ lam, double* __restrict__ G, double cl,
                                  double cg, double cs, double* __restrict__ a_next, double* __restrict__ out,
                                  double* __restrict__ sbar) {
  const Pad P = pad_of(g, bc);
  const long long n = g.cells * g.batch;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / g.cells, r = i - b * g.cells;
    const int z = (int)(r / g.plane);
    const long long rr = r - (long long)z * g.plane;
    const int y = (int)(rr / g.nx), x = (int)(rr - (long long)y * g.nx);
    const long long boxp = b * 5 * P.cellsp + (long long)z * P.planep;
    auto atp = [&](int xp, int yp) { return boxp + (long long)yp * P.nxp + xp; };
    auto wget = [&](long long o, double v[5]) {
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = (double)W[o + k * P.cellsp];
    };
    auto gget = [&](long long o, double v[5]) {
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] = gp[o + k * P.cellsp];
    };
    const int xp = x + P.ix, yp = y + P.iy;
    double gc[5], h[5], d[5], wc[5];
    gget(atp(xp, yp), gc);
    // wall rows first: a ghost row's output goes to the row it was built from
    if (P.iy && (y == 0 || y == g.ny - 1)) {
      for (int side = 0; side < 2; ++side) {
        if ((side == 0 && y != 0) || (side == 1 && y != g.ny - 1)) continue;
        gget(atp(xp, side == 0 ? 0 : P.nyp - 1), h);
        wget(atp(xp, yp), wc);
        ghost_pullback(wc, 1, side, bc, h, d);
#pragma unroll
        for (int k = 0; k < 5; ++k) gc[k] += d[k];
      }
    }
    // then the inflow and outflow columns: each column ghost's output, with its wall
    // ghosts' outputs pulled back onto it at the first and last rows
    if (P.ix && (x == 0 || x == g.nx - 1)) {
      for (int side = 0; side < 2; ++side) {
        if ((side == 0 && x != 0) || (side == 1 && x != g.nx - 1)) continue;
        const int xg = side == 0 ? 0 : P.nxp - 1;
        gget(atp(xg, yp), h);
        if (P.iy && (y == 0 || y == g.ny - 1)) {
          for (int ws = 0; ws < 2; ++ws) {
            if ((ws == 0 && y != 0) || (ws == 1 && y != g.ny - 1)) continue;
            double hc[5], dc[5], wg[5];
            gget(atp(xg, ws == 0 ? 0 : P.nyp - 1), hc);
            wget(atp(xg, yp), wg);   // the column ghost the corner was built from
            ghost_pullback(wg, 1, ws, bc, hc, dc);
#pragma unroll
            for (int k = 0; k < 5; ++k) h[k] += dc[k];
          }
        }
        wget(atp(xp, yp), wc);
        ghost_pullback(wc, 0, side, bc, h, d);
#pragma unroll
        for (int k = 0; k < 5; ++k) gc[k] += d[k];
      }
    }
    // the seed of this stage and the added viscosity with closed boundary faces
    const long long o = b * 5 * g.cells + r;
    double a[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) a[k] = sa * A[o + k * g.cells];
    if (nu) {
      const long long c0 = b * g.cells + r;
      const double nc = (double)nu[c0];
      const int xm = x == 0 ? g.nx - 1 : x - 1, xq = x == g.nx - 1 ? 0 : x + 1;
      const int ym = y == 0 ? g.ny - 1 : y - 1, yq = y == g.ny - 1 ? 0 : y + 1;
      const int zm = z == 0 ? g.nz - 1 : z - 1, zq = z == g.nz - 1 ? 0 : z + 1;
      const bool cxm = P.ix && x == 0, cxq = P.ix && x == g.nx - 1;   // closed faces
      const bool cym = P.iy && y == 0, cyq = P.iy && y == g.ny - 1;
      const long long bb = b * g.cells;
      const long long oxm = (long long)z * g.plane + (long long)y * g.nx + xm;
      const long long oxq = (long long)z * g.plane + (long long)y * g.nx + xq;
      const long long oym = (long long)z * g.plane + (long long)ym * g.nx + x;
      const long long oyq = (long long)z * g.plane + (long long)yq * g.nx + x;
      const long long ozm = (long long)zm * g.plane + (long long)y * g.nx + x;
      const long long ozq = (long long)zq * g.plane + (long long)y * g.nx + x;
      const double fxm = cxm ? 0.0 : 0.5 * (nc + (double)nu[bb + oxm]);
      const double fxq = cxq ? 0.0 : 0.5 * (nc + (double)nu[bb + oxq]);
      const double fym = cym ? 0.0 : 0.5 * (nc + (double)nu[bb + oym]);
      const double fyq = cyq ? 0.0 : 0.5 * (nc + (double)nu[bb + oyq]);
      const double fzm = 0.5 * (nc + (double)nu[bb + ozm]);
      const double fzq = 0.5 * (nc + (double)nu[bb + ozq]);
      const long long ab = b * 5 * g.cells;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const double* Ak = A + ab + (long long)k * g.cells;
        const double ac = a[k];
        const double L = (fxq * (sa * Ak[oxq] - ac) - fxm * (ac - sa * Ak[oxm])) * i2x +
                         (fyq * (sa * Ak[oyq] - ac) - fym * (ac - sa * Ak[oym])) * i2y +
                         (fzq * (sa * Ak[ozq] - ac) - fzm * (ac - sa * Ak[ozm])) * i2z;
        gc[k] += (k == 0 ? nus0 : (k == 4 ? nus2 : nus1)) * L;
      }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const long long ok = o + (long long)k * g.cells;
      if (mode == 0) {
        out[ok] = gc[k];
        continue;
      }
      const double Gs = (first ? 0.0 : G[ok]) + gc[k];
      if (last) {
        out[ok] = lam[ok] + Gs;
      } else {
        G[ok] = Gs;
        a_next[ok] = cl * lam[ok] + cg * gc[k] + cs * Gs;
      }
      if (sbar) sbar[ok] += a[k];
    }
  }
}

constexpr int BB = 256;

unsigned blocks_for(long long n) {
  long long b = (n + BB - 1) / BB;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b > 0 ? b : 1);
}

}  // namespace

long long bc_padded_cells(const GridDesc& g, const BcDesc& bc) {
  return (long long)(g.nx + 2 * bc.inout) * (g.ny + 2 * bc.walls) * g.nz;
}

template <class TO, class TI>
cudaError_t launch_bc_embed(const GridDesc& g, const BcDesc& bc, int ncomp, double scale, const TI* src, TO* dst,
                            cudaStream_t st) {
  const long long n = bc_padded_cells(g, bc) * ncomp * g.batch;
  k_bc_embed<TO, TI><<<blocks_for(n), BB, 0, st>>>(g, bc, ncomp, scale, src, dst);
  count_launch();
  return cudaGetLastError();
}

template <class TO, class TI>
cudaError_t launch_bc_crop(const GridDesc& g, const BcDesc& bc, int ncomp, const TI* src, TO* dst, cudaStream_t st) {
  const long long n = g.cells * ncomp * g.batch;
  k_bc_crop<TO, TI><<<blocks_for(n), BB, 0, st>>>(g, bc, ncomp, src, dst);
  count_launch();
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_bc_ghosts(const GridDesc& g, const BcDesc& bc, T* W, cudaStream_t st) {
  const long long per = (long long)((bc.inout ? 2 * g.ny : 0) + (bc.walls ? 2 * (g.nx + 2 * bc.inout) : 0)) * g.nz;
  k_bc_ghosts<T><<<blocks_for(per * g.batch), BB, 0, st>>>(g, bc, W);
  count_launch();
  return cudaGetLastError();
}

template <class CT, class NU>
cudaError_t launch_bc_adj_epilogue(const GridDesc& g, const BcDesc& bc, const BcEpilogue& e, const double* gp,
                                   const CT* W, const NU* nu, cudaStream_t st) {
  k_bc_adj_epilogue<CT, NU><<<blocks_for(g.cells * g.batch), BB, 0, st>>>(
      g, bc, gp, W, e.A, e.sa, nu, e.nus[0], e.nus[1], e.nus[2], e.i2[0], e.i2[1], e.i2[2], e.mode, e.first, e.last,
      e.lam, e.G, e.cl, e.cg, e.cs, e.a_next, e.out, e.sbar);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_bc_embed<double, double>(const GridDesc&, const BcDesc&, int, double, const double*,
                                                     double*, cudaStream_t);
template cudaError_t launch_bc_embed<float, double>(const GridDesc&, const BcDesc&, int, double, const double*,
                                                    float*, cudaStream_t);
template cudaError_t launch_bc_crop<double, double>(const GridDesc&, const BcDesc&, int, const double*, double*,
                                                    cudaStream_t);
template cudaError_t launch_bc_crop<float, float>(const GridDesc&, const BcDesc&, int, const float*, float*,
                                                  cudaStream_t);
template cudaError_t launch_bc_ghosts<double>(const GridDesc&, const BcDesc&, double*, cudaStream_t);
template cudaError_t launch_bc_ghosts<float>(const GridDesc&, const BcDesc&, float*, cudaStream_t);
template cudaError_t launch_bc_adj_epilogue<double, float>(const GridDesc&, const BcDesc&, const BcEpilogue&,
                                                           const double*, const double*, const float*, cudaStream_t);
template cudaError_t launch_bc_adj_epilogue<double, double>(const GridDesc&, const BcDesc&, const BcEpilogue&,
                                                            const double*, const double*, const double*, cudaStream_t);
template cudaError_t launch_bc_adj_epilogue<float, float>(const GridDesc&, const BcDesc&, const BcEpilogue&,
                                                          const double*, const float*, const float*, cudaStream_t);

}  // namespace ns
