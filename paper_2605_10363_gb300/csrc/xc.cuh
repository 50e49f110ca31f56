// Exchange-correlation energy density f(rho, sigma) and its analytic
// derivatives v_rho = df/drho, v_sigma = df/dsigma, in FP64, spin-restricted.
//
// LDA exchange (Slater): f = -C_x rho^(4/3), C_x = (3/4)(3/pi)^(1/3).
// PBE exchange: f = f_LDA F(s2), F = 1 + kappa - kappa/(1 + mu s2/kappa),
//   s2 = sigma / (4 (3 pi^2)^(2/3) rho^(8/3)), kappa = 0.804, mu = beta pi^2/3.
// PBE correlation on PW92: f = rho (eps(rs) + H(eps, y)), rs = (3/(4 pi rho))^(1/3),
//   eps = -2A(1 + a1 rs) ln(1 + 1/Q), Q = 2A(b1 rs^(1/2) + b2 rs + b3 rs^(3/2) + b4 rs^2),
//   y = t^2 = sigma pi / (16 (3 pi^2)^(1/3) rho^(7/3)),
//   H = gamma ln(1 + G), G = (beta/gamma) y (1 + B y) / (1 + B y + B^2 y^2),
//   B = (beta/gamma) / (exp(-eps/gamma) - 1), gamma = (1 - ln 2)/pi^2.
// Derivatives used below (derived by hand):
//   dG/dy = (beta/gamma)(1 + 2 B y) / den^2,  den = 1 + B y + B^2 y^2
//   dG/dB = -(beta/gamma) B y^3 (2 + B y) / den^2
//   dB/deps = B^2 exp(-eps/gamma) / beta
//   deps/drs = -2 A a1 ln(1 + 1/Q) + 2A(1 + a1 rs) Q' / (Q^2 + Q)
//   drs/drho = -rs/(3 rho),  dy/drho = -(7/3) y / rho,  ds2/drho = -(8/3) s2 / rho.
#pragma once

namespace kldi {

struct XcOut {
  double f, vr, vs;
};

__host__ __device__ inline XcOut xc_lda_x(double rho) {
  const double cx = 0.73855876638202240587;  // (3/4)(3/pi)^(1/3)
  const double r13 = cbrt(rho);
  XcOut o;
  o.f = -cx * rho * r13;
  o.vr = -(4.0 / 3.0) * cx * r13;
  o.vs = 0.0;
  return o;
}

__host__ __device__ inline XcOut xc_pbe(double rho, double sigma) {
  const double kPi = 3.14159265358979323846;
  const double kappa = 0.804;
  const double beta = 0.06672455060314922;
  const double mu = beta * kPi * kPi / 3.0;
  const double gamma = (1.0 - 0.69314718055994530942) / (kPi * kPi);
  const double A = 0.031091, a1 = 0.21370;
  const double b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
  if (sigma < 0.0) sigma = 0.0;

  // exchange
  const XcOut lda = xc_lda_x(rho);
  const double r13 = cbrt(rho);
  const double rho83 = rho * rho * r13 * r13;                  // rho^(8/3)
  const double c_s = 1.0 / (4.0 * cbrt(9.0 * kPi * kPi * kPi * kPi));  // 1/(4 (3 pi^2)^(2/3))
  const double s2 = sigma * c_s / rho83;
  const double qx = 1.0 + mu * s2 / kappa;
  const double F = 1.0 + kappa - kappa / qx;
  const double dF = mu / (qx * qx);                            // dF/ds2
  const double fx = lda.f * F;
  const double vrx = lda.vr * F + lda.f * dF * (-(8.0 / 3.0) * s2 / rho);
  const double vsx = lda.f * dF * c_s / rho83;

  // correlation
  const double rs = cbrt(3.0 / (4.0 * kPi * rho));
  const double srs = sqrt(rs);
  const double Q = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
  const double dQ = 2.0 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs);
  const double L = log1p(1.0 / Q);
  const double eps = -2.0 * A * (1.0 + a1 * rs) * L;
  const double deps_drs = -2.0 * A * a1 * L + 2.0 * A * (1.0 + a1 * rs) * dQ / (Q * Q + Q);
  const double c_t = kPi / (16.0 * cbrt(3.0 * kPi * kPi));
  const double y = sigma * c_t / (rho * rho * r13);           // t^2 = sigma c_t rho^(-7/3)
  const double E = exp(-eps / gamma);
  const double Bc = (beta / gamma) / (E - 1.0);
  const double den = 1.0 + Bc * y + Bc * Bc * y * y;
  const double G = (beta / gamma) * y * (1.0 + Bc * y) / den;
  const double H = gamma * log1p(G);
  const double dG_dy = (beta / gamma) * (1.0 + 2.0 * Bc * y) / (den * den);
  const double dG_dB = -(beta / gamma) * Bc * y * y * y * (2.0 + Bc * y) / (den * den);
  const double dB_deps = Bc * Bc * E / beta;
  const double dH_dy = gamma * dG_dy / (1.0 + G);
  const double dH_deps = gamma * dG_dB * dB_deps / (1.0 + G);
  const double drs_drho = -rs / (3.0 * rho);
  const double dy_drho = -(7.0 / 3.0) * y / rho;
  const double deps_drho = deps_drs * drs_drho;
  const double fc = rho * (eps + H);
  const double vrc = (eps + H) + rho * (deps_drho + dH_deps * deps_drho + dH_dy * dy_drho);
  const double vsc = rho * dH_dy * c_t / (rho * rho * r13);

  XcOut o;
  o.f = fx + fc;
  o.vr = vrx + vrc;
  o.vs = vsx + vsc;
  return o;
}

}  // namespace kldi
