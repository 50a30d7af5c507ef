// Roe dissipation of one face (section "Numerical methods": the approximate Roe solver
// of the paper's flow solver) and its hand-reversed adjoint, in the primitive variables
// (rho, u1, u2, u3, e) the stencil kernels keep in shared memory.
//
// For a face with normal e_D between cells L and R:
//   Roe state: sqrt(rho)-weighted means u~, H~ (H = gamma e + |u|^2/2), rho~ =
//   sqrt(rho_L rho_R), c~^2 = (gamma-1)(H~ - |u~|^2/2);
//   wave strengths a1,3 = (dp -+ rho~ c~ du_D) / (2 c~^2), a2 = drho - dp / c~^2 and the
//   shear jumps rho~ (du - du_D e_D);
//   speeds u~_D - c~, u~_D, u~_D + c~ with Harten's entropy fix
//   |lam| -> (lam^2 + delta^2) / (2 delta) where |lam| < delta, delta = roe_delta c~;
//   D = (sum_k |lam_k| a_k r_k) / 2 with the eigenvectors r_k of the Euler Jacobian at
//   the Roe state.  The face flux is Phi = (F_L + F_R)/2 - D - F^v.
//
// roe_dissipation_adj returns the adjoints of the two cells' primitives for a given
// adjoint of D: every forward step reversed, last first.
#pragma once

#include "ns_common.cuh"

namespace ns {

__device__ __forceinline__ float sq_root(float x) { return sqrtf(x); }
__device__ __forceinline__ double sq_root(double x) { return sqrt(x); }
__device__ __forceinline__ Dual sq_root(Dual x) {
  const double r = sqrt(x.v);
  return Dual(r, x.d / (2.0 * r));
}

// |x| with Harten's entropy fix; the branch is taken on the value.
template <class CT>
__device__ __forceinline__ CT abs_fix(CT x, CT dl) {
  const double xv = (double)val(x), dv = (double)val(dl);
  if (fabs(xv) < dv) return (x * x + dl * dl) / (CT(2) * dl);
  return xv >= 0.0 ? x : CT(0) - x;
}

// derivatives of abs_fix with respect to x and delta
template <class CT>
__device__ __forceinline__ void abs_fix_d(CT x, CT dl, CT& fx, CT& fd) {
  if (fabs((double)val(x)) < (double)val(dl)) {
    fx = x / dl;
    fd = (dl * dl - x * x) / (CT(2) * dl * dl);
  } else {
    fx = (double)val(x) >= 0.0 ? CT(1) : CT(-1);
    fd = CT(0);
  }
}

// Roe-state quantities shared by the forward and the reverse pass.
template <int D, class CT>
struct RoeState {
  CT pL, pR, HL, HR, sL, sR, inv, wl, wr, ut[3], Ht, rt, q2, c2, c, ic2, un;
  CT dr, dp, du[3], dun, A, h, a1, a2, a3, dl, l1, l2, l3, W1, W2, W3, Sg, S, Dif, udu;

  __device__ __forceinline__ RoeState(const Coef<CT>& k, const CT* qL, const CT* qR) {
    const CT g = k.gamma, gm1 = k.gm1;
    pL = gm1 * qL[0] * qL[4];
    pR = gm1 * qR[0] * qR[4];
    HL = g * qL[4] + CT(0.5) * (qL[1] * qL[1] + qL[2] * qL[2] + qL[3] * qL[3]);
    HR = g * qR[4] + CT(0.5) * (qR[1] * qR[1] + qR[2] * qR[2] + qR[3] * qR[3]);
    sL = sq_root(qL[0]);
    sR = sq_root(qR[0]);
    inv = CT(1) / (sL + sR);
    wl = sL * inv;
    wr = sR * inv;
#pragma unroll
    for (int j = 0; j < 3; ++j) ut[j] = wl * qL[1 + j] + wr * qR[1 + j];
    Ht = wl * HL + wr * HR;
    rt = sL * sR;
    q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
    c2 = gm1 * (Ht - CT(0.5) * q2);
    c = sq_root(c2);
    ic2 = CT(1) / c2;
    un = ut[D];
    dr = qR[0] - qL[0];
    dp = pR - pL;
#pragma unroll
    for (int j = 0; j < 3; ++j) du[j] = qR[1 + j] - qL[1 + j];
    dun = du[D];
    A = rt * c * dun;
    h = CT(0.5) * ic2;
    a1 = (dp - A) * h;
    a2 = dr - dp * ic2;
    a3 = (dp + A) * h;
    dl = k.roe_delta * c;
    l1 = abs_fix(un - c, dl);
    l2 = abs_fix(un, dl);
    l3 = abs_fix(un + c, dl);
    W1 = l1 * a1;
    W2 = l2 * a2;
    W3 = l3 * a3;
    Sg = l2 * rt;
    S = W1 + W2 + W3;
    Dif = W3 - W1;
    udu = ut[0] * du[0] + ut[1] * du[1] + ut[2] * du[2];
  }
};

template <int D, class CT>
__device__ __forceinline__ void roe_dissipation(const Coef<CT>& k, const CT* qL, const CT* qR, CT Dv[5]) {
  const RoeState<D, CT> r(k, qL, qR);
  const CT half = CT(0.5);
  Dv[0] = half * r.S;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    Dv[1 + j] = half * (r.S * r.ut[j] + (j == D ? r.c * r.Dif : r.Sg * r.du[j]));
  Dv[4] = half * ((r.W1 + r.W3) * r.Ht + r.c * r.un * r.Dif + r.W2 * half * r.q2 +
                  r.Sg * (r.udu - r.un * r.dun));
}

// bL, bR: adjoints of (rho, u1, u2, u3, e) of the left and right cell for the adjoint
// Db of the dissipation D.
template <int D, class CT>
__device__ __forceinline__ void roe_dissipation_adj(const Coef<CT>& k, const CT* qL, const CT* qR,
                                                    const CT Db[5], CT bL[5], CT bR[5]) {
  const RoeState<D, CT> r(k, qL, qR);
  const CT gm1 = k.gm1, half = CT(0.5);
  CT b[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) b[v] = half * Db[v];
  // D0 = S; D_j = S ut_j + (j == D ? c Dif : Sg du_j)
  CT Sb = b[0], utb[3], dub[3], Sgb = CT(0), cb = CT(0), Difb = CT(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    Sb = Sb + b[1 + j] * r.ut[j];
    utb[j] = b[1 + j] * r.S;
    dub[j] = CT(0);
    if (j == D) {
      cb = cb + b[1 + j] * r.Dif;
      Difb = Difb + b[1 + j] * r.c;
    } else {
      Sgb = Sgb + b[1 + j] * r.du[j];
      dub[j] = b[1 + j] * r.Sg;
    }
  }
  // D4 = (W1 + W3) Ht + c un Dif + W2 q2/2 + Sg (udu - un dun)
  CT W1b = b[4] * r.Ht, W3b = b[4] * r.Ht, W2b = b[4] * half * r.q2;
  CT Htb = b[4] * (r.W1 + r.W3);
  cb = cb + b[4] * r.un * r.Dif;
  CT unb = b[4] * r.c * r.Dif - b[4] * r.Sg * r.dun;
  Difb = Difb + b[4] * r.c * r.un;
  CT q2b = b[4] * half * r.W2;
  Sgb = Sgb + b[4] * (r.udu - r.un * r.dun);
  const CT udub = b[4] * r.Sg;
  CT dunb = CT(0) - b[4] * r.Sg * r.un;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    utb[j] = utb[j] + udub * r.du[j];
    dub[j] = dub[j] + udub * r.ut[j];
  }
  // S = W1 + W2 + W3, Dif = W3 - W1, Sg = l2 rt, W_i = l_i a_i
  W1b = W1b + Sb - Difb;
  W2b = W2b + Sb;
  W3b = W3b + Sb + Difb;
  const CT l1b = W1b * r.a1, l2b = W2b * r.a2 + Sgb * r.rt, l3b = W3b * r.a3;
  const CT a1b = W1b * r.l1, a2b = W2b * r.l2, a3b = W3b * r.l3;
  CT rtb = Sgb * r.l2;
  // l1 = fix(un - c), l2 = fix(un), l3 = fix(un + c), dl = roe_delta c
  CT fx, fd, dlb;
  abs_fix_d(r.un - r.c, r.dl, fx, fd);
  unb = unb + l1b * fx;
  cb = cb - l1b * fx;
  dlb = l1b * fd;
  abs_fix_d(r.un, r.dl, fx, fd);
  unb = unb + l2b * fx;
  dlb = dlb + l2b * fd;
  abs_fix_d(r.un + r.c, r.dl, fx, fd);
  unb = unb + l3b * fx;
  cb = cb + l3b * fx;
  dlb = dlb + l3b * fd;
  cb = cb + k.roe_delta * dlb;
  // a1 = (dp - A) h, a2 = dr - dp ic2, a3 = (dp + A) h, h = ic2 / 2, ic2 = 1 / c2
  const CT dpb = (a1b + a3b) * r.h - a2b * r.ic2;
  const CT Ab = (a3b - a1b) * r.h;
  const CT hb = a1b * (r.dp - r.A) + a3b * (r.dp + r.A);
  const CT drb = a2b;
  const CT ic2b = half * hb - a2b * r.dp;
  CT c2b = CT(0) - ic2b * r.ic2 * r.ic2;
  // A = rt c dun
  rtb = rtb + Ab * r.c * r.dun;
  cb = cb + Ab * r.rt * r.dun;
  dunb = dunb + Ab * r.rt * r.c;
  utb[D] = utb[D] + unb;
  dub[D] = dub[D] + dunb;
  // c = sqrt(c2), c2 = (gamma-1)(Ht - q2/2), q2 = |ut|^2
  c2b = c2b + cb / (CT(2) * r.c);
  Htb = Htb + gm1 * c2b;
  q2b = q2b - half * gm1 * c2b;
#pragma unroll
  for (int j = 0; j < 3; ++j) utb[j] = utb[j] + CT(2) * r.ut[j] * q2b;
  // Ht = wl HL + wr HR, ut = wl uL + wr uR, rt = sL sR, wl = sL inv, wr = sR inv
  const CT HLb = r.wl * Htb, HRb = r.wr * Htb;
  CT wlb = r.HL * Htb, wrb = r.HR * Htb;
  CT uLb[3], uRb[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    uLb[j] = r.wl * utb[j];
    uRb[j] = r.wr * utb[j];
    wlb = wlb + qL[1 + j] * utb[j];
    wrb = wrb + qR[1 + j] * utb[j];
  }
  CT sLb = r.sR * rtb + r.inv * wlb, sRb = r.sL * rtb + r.inv * wrb;
  const CT invb = r.sL * wlb + r.sR * wrb;
  sLb = sLb - r.inv * r.inv * invb;
  sRb = sRb - r.inv * r.inv * invb;
  CT rLb = sLb / (CT(2) * r.sL) - drb, rRb = sRb / (CT(2) * r.sR) + drb;
  // dp = pR - pL, du = uR - uL, H = gamma e + |u|^2/2, p = (gamma-1) rho e
  const CT pLb = CT(0) - dpb, pRb = dpb;
  CT eLb = k.gamma * HLb + gm1 * qL[0] * pLb, eRb = k.gamma * HRb + gm1 * qR[0] * pRb;
  rLb = rLb + gm1 * qL[4] * pLb;
  rRb = rRb + gm1 * qR[4] * pRb;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    uLb[j] = uLb[j] - dub[j] + qL[1 + j] * HLb;
    uRb[j] = uRb[j] + dub[j] + qR[1 + j] * HRb;
  }
  bL[0] = rLb;
  bR[0] = rRb;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    bL[1 + j] = uLb[j];
    bR[1 + j] = uRb[j];
  }
  bL[4] = eLb;
  bR[4] = eRb;
}

}  // namespace ns
