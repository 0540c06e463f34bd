// fforce.cu -- the fermion force (Sec. 2.2: "by means of the identity
// dD^-1 = -D^-1 (dD) D^-1 the fermion force can be evaluated"; only the hopping
// term depends on U) for S_pf = phi^+ (Mhat^+ Mhat)^-1 phi on the even sites.
//
// With X = (Mhat^+ Mhat)^-1 phi and Y = Mhat X,
//   dS = -2 Re[Y^+ dMhat X],  dMhat = -kappa^2 (dH_eo A_o^-1 H_oe + H_eo A_o^-1 dH_oe),
// so dS = 2 kappa^2 Re[Lf^+ dH Rf] with full-lattice fields
//   Lf = (Y_e, W_o),  W_o = A_o^-+ (H^+)_oe Y_e,
//   Rf = (X_e, Z_o),  Z_o = A_o^-1 H_oe X_e.
// For the link U_mu(x) -> exp(i w^a T^a) U_mu(x):
//   dS/dw^a = -2 kappa^2 bc Im Tr[T^a (C1 - C2)],
//   C1 = sum_spin (U Rf(x+mu)) (x) ((1 - g_mu) Lf(x))^+
//   C2 = sum_spin Rf(x) (x) (U (1 + g_mu) Lf(x+mu))^+.
// Because (1 -+ g_mu) = 2 P-+ with P a rank-2 projector, each spin sum reduces
// to two colour outer products of spin-projected half spinors:
//   C1 = sum_{k=0,1} (U hR_k) hL_k^+,  hR = proj+(Rf(x+mu)), hL = proj+(Lf(x))
//   C2 = sum_{k=0,1} h'R_k (U h'L_k)^+, h'R = proj-(Rf(x)),   h'L = proj-(Lf(x+mu))
// where proj_s(psi) = psi_up - s B psi_dn (gamma_mu = [[0,B],[B^+,0]]).
// One thread per site computes the four links of that site (FP64), reading
// 18-real links or, for a field imported with recon = 12, 12-real links with
// the third row rebuilt (the paper suggests REC12 for this kernel too).
#include "internal.h"

namespace lqcd {

using C = Cx<double>;

template <int MU, int S>
LQCD_DEV void proj(const C ps[12], C h[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const C p0 = ps[c], p1 = ps[3 + c], p2 = ps[6 + c], p3 = ps[9 + c];
    if (MU == 0) {
      h[c] = S > 0 ? p0 + times_i(p3) : p0 - times_i(p3);
      h[3 + c] = S > 0 ? p1 + times_i(p2) : p1 - times_i(p2);
    } else if (MU == 1) {
      h[c] = S > 0 ? p0 + p3 : p0 - p3;
      h[3 + c] = S > 0 ? p1 - p2 : p1 + p2;
    } else if (MU == 2) {
      h[c] = S > 0 ? p0 + times_i(p2) : p0 - times_i(p2);
      h[3 + c] = S > 0 ? p1 - times_i(p3) : p1 + times_i(p3);
    } else {
      h[c] = S > 0 ? p0 - p2 : p0 + p2;
      h[3 + c] = S > 0 ? p1 - p3 : p1 + p3;
    }
  }
}

LQCD_DEV void load12(const double2 *f, int Vh, int p, int cb, C s[12]) {
  const double2 *b = f + (size_t)p * 12 * Vh;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    double2 w = b[(size_t)k * Vh + cb];
    s[k] = {w.x, w.y};
  }
}

template <int MU, int RECON>
LQCD_DEV void link_force(const GaugeView &U, const double2 *Lf, const double2 *Rf, const Geom &g, const Site &s,
                         int p, int cb, long lexi, double pref, double *out) {
  const int j = neighbour_cb(g, s, MU, +1);
  C u[9];
  LinkIO<LQCD_F64, RECON>::load(U, p, MU, cb, u);
  if (RECON == 12) reconstruct_row2(u);  // Sec. 4.1 applied to the force (the paper's outlook)
  C a[12], hR[6], hL[6], hR2[6], hL2[6];
  load12(Rf, g.Vh, p ^ 1, j, a);
  proj<MU, 1>(a, hR);
  load12(Lf, g.Vh, p, cb, a);
  proj<MU, 1>(a, hL);
  load12(Rf, g.Vh, p, cb, a);
  proj<MU, -1>(a, hR2);
  load12(Lf, g.Vh, p ^ 1, j, a);
  proj<MU, -1>(a, hL2);
  // U hR and U h'L
  C uR[6], uL[6];
#pragma unroll
  for (int k = 0; k < 2; k++)
#pragma unroll
    for (int r = 0; r < 3; r++) {
      C s1 = u[3 * r] * hR[3 * k], s2 = u[3 * r] * hL2[3 * k];
      s1 = cmadd(u[3 * r + 1], hR[3 * k + 1], s1);
      s2 = cmadd(u[3 * r + 1], hL2[3 * k + 1], s2);
      s1 = cmadd(u[3 * r + 2], hR[3 * k + 2], s1);
      s2 = cmadd(u[3 * r + 2], hL2[3 * k + 2], s2);
      uR[3 * k + r] = s1;
      uL[3 * k + r] = s2;
    }
  // D = C1 - C2, D_cd = sum_k uR_kc conj(hL_kd) - hR2_kc conj(uL_kd)
  C D[9];
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int d = 0; d < 3; d++) {
      C t = czero<double>();
#pragma unroll
      for (int k = 0; k < 2; k++) {
        t = cmadd(uR[3 * k + c], conj(hL[3 * k + d]), t);
        t = t - hR2[3 * k + c] * conj(uL[3 * k + d]);
      }
      D[3 * c + d] = t;
    }
  // Im Tr(lambda^a D)
  double tr[8];
  tr[0] = (D[3] + D[1]).im;
  tr[1] = times_i(D[1] - D[3]).im;
  tr[2] = (D[0] - D[4]).im;
  tr[3] = (D[6] + D[2]).im;
  tr[4] = times_i(D[2] - D[6]).im;
  tr[5] = (D[7] + D[5]).im;
  tr[6] = times_i(D[5] - D[7]).im;
  tr[7] = (D[0] + D[4] - D[8] - D[8]).im * 0.57735026918962576451;
  const double bc = (MU == 3 && g.antiper && s.t == g.L[3] - 1) ? -1.0 : 1.0;
  const long V = 2L * g.Vh;
  double *o = out + ((size_t)MU * V + lexi) * 8;
  // -2 kappa^2 bc Im Tr[T^a D] = -kappa^2 bc Im Tr[lambda^a D]
#pragma unroll
  for (int k = 0; k < 8; k++) o[k] = -pref * bc * tr[k];
}

template <int RECON>
__global__ void __launch_bounds__(128) fermion_force_kernel(GaugeView U, const double2 *Lf, const double2 *Rf,
                                                            Geom g, double pref, double *out) {
  long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= 2L * g.Vh) return;
  int p = (int)(tid / g.Vh), cb = (int)(tid - (long)p * g.Vh);
  Site s = site_of(g, p, cb);
  long lexi = lexi_index(g, s);
  link_force<0, RECON>(U, Lf, Rf, g, s, p, cb, lexi, pref, out);
  link_force<1, RECON>(U, Lf, Rf, g, s, p, cb, lexi, pref, out);
  link_force<2, RECON>(U, Lf, Rf, g, s, p, cb, lexi, pref, out);
  link_force<3, RECON>(U, Lf, Rf, g, s, p, cb, lexi, pref, out);
}

// dS/dw into out [4][V][8] from EO full F64 fields Lf, Rf; pref = kappa^2.
// Uv: the FP64 links in format recon (18, or 12 with the third row rebuilt).
lqcd_status fermion_force_raw(lqcd_ctx *ctx, const lqcd_gauge *U, const GaugeView &Uv, int recon, const void *Lf,
                              const void *Rf, double kappa, double *out) {
  long V = 2L * U->g.Vh;
  const unsigned grid = (unsigned)((V + 127) / 128);
  if (recon == 12)
    fermion_force_kernel<12><<<grid, 128, 0, ctx->stream>>>(Uv, (const double2 *)Lf, (const double2 *)Rf, U->g,
                                                            kappa * kappa, out);
  else
    fermion_force_kernel<18><<<grid, 128, 0, ctx->stream>>>(Uv, (const double2 *)Lf, (const double2 *)Rf, U->g,
                                                            kappa * kappa, out);
  LQCD_CUDA(ctx, cudaGetLastError());
  return LQCD_OK;
}

}  // namespace lqcd
