// Device-side Milne-Eddington synthesis for sm_103a: Voigt/Faraday-Voigt
// functions, absorption matrix of a normal Zeeman triplet, closed-form
// Unno-Rachkovsky solution and its analytic derivatives, fused with the
// filter convolution.  All arithmetic in FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vfisv {

// Number of terms of the Weideman (1994) rational series for w(z).  With 16
// terms the truncation error is below 1.3e-7 for Im z >= 0, about the size
// of the FP32 rounding error of the evaluation itself.
constexpr int kWeidN = 16;
// Unroll factor of the Horner loop (15 = fully unrolled); a smaller factor
// shrinks the wavelength loop's code at the cost of loop overhead.
#ifndef VFISV_HORNER_UNROLL
#define VFISV_HORNER_UNROLL 15
#endif
constexpr int kHornerUnroll = VFISV_HORNER_UNROLL;
// 1: multiply the filter weights by 1/Delta once per wavelength (6 products,
// 6 live registers); 0: scale the six derivative row values instead.
#ifndef VFISV_FOLD_ID_IN_WEIGHTS
#define VFISV_FOLD_ID_IN_WEIGHTS 1
#endif
constexpr float kInvSqrtPi = 0.56418958354775628695f;
constexpr float kTwoInvSqrtPi = 1.1283791670955125739f;
constexpr float kDeg = 0.017453292519943295769f;

// Coefficients of w(z) ~ 1/(sqrt(pi) (L - iz)) + 2/(L - iz)^2 sum_{n=0}^{N-1} a_{n+1} Z^n,
// Z = (L + iz)/(L - iz): a_n are the Fourier coefficients of
// (L^2 + t^2) exp(-t^2) in the angle theta with t = L tan(theta/2).
// Filled on the host (api.cu) and passed by value into kernel parameters.
struct Weideman {
  float L;
  float a[kWeidN + 1];  // a[1..N] used
};

// Line constants in the units the kernels use (mA, gauss, km/s).
struct LineK {
  float cB;  // Zeeman shift per gauss, Eq. 7: 4.66685e-10 g lambda0^2
  float cv;  // Doppler shift per km/s: lambda0 / c
  float mu;
};

// Reciprocal with at most 1 ulp error (PTX rcp.approx); the operands here
// are normal numbers well away from the flush-to-zero range.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// H(a,u) + i F(a,u) = w(u + i a) for a >= 0 (Sec. 3.2).
__device__ __forceinline__ void faddeeva(const Weideman& W, float u, float a,
                                         float& H, float& F) {
  const float L = W.L;
  const float lp = L + a;
  const float d = fmaf(lp, lp, u * u);
  const float rd = rcp_fast(d);
  const float zr = fmaf(L - a, lp, -u * u) * rd;
  const float zi = (2.0f * L * u) * rd;
  float pr = W.a[kWeidN], pi = 0.0f;
#pragma unroll kHornerUnroll
  for (int n = kWeidN - 1; n >= 1; --n) {
    const float t = fmaf(pr, zr, fmaf(-pi, zi, W.a[n]));
    pi = fmaf(pr, zi, pi * zr);
    pr = t;
  }
  const float qr = lp * rd, qi = u * rd;  // 1/(L - iz)
  const float q2r = fmaf(qr, qr, -qi * qi), q2i = 2.0f * qr * qi;
  H = fmaf(2.0f, fmaf(pr, q2r, -pi * q2i), kInvSqrtPi * qr);
  F = fmaf(2.0f, fmaf(pr, q2i, pi * q2r), kInvSqrtPi * qi);
}

// Model bounds, applied after every step of the inversion and to initial
// models: B < 0 -> (-B, 180 - gamma), gamma reflected into [0, 180], psi
// mod 180, then the box limits.
__device__ __forceinline__ void apply_bounds(float (&m)[10]) {
  if (m[0] < 0.0f) {
    m[0] = -m[0];
    m[1] = 180.0f - m[1];
  }
  float g = fmodf(m[1], 360.0f);
  if (g < 0.0f) g += 360.0f;
  m[1] = (g > 180.0f) ? 360.0f - g : g;
  float ps = fmodf(m[2], 180.0f);
  if (ps < 0.0f) ps += 180.0f;
  if (ps >= 180.0f) ps = 0.0f;
  m[2] = ps;
  m[0] = fminf(m[0], 6000.0f);
  m[3] = fminf(fmaxf(m[3], 0.01f), 500.0f);
  m[4] = fminf(fmaxf(m[4], 5.0f), 150.0f);
  m[5] = fminf(fmaxf(m[5], 0.0f), 5.0f);
  m[6] = fminf(fmaxf(m[6], -20.0f), 20.0f);
  m[7] = fminf(fmaxf(m[7], 0.0f), 2.0f);
  m[8] = fminf(fmaxf(m[8], 0.0f), 2.0f);
}

// Per-pixel constants of one synthesis.
struct PixK {
  float invD;   // 1 / dlambdaD
  float uv;     // Doppler shift / dlambdaD
  float uB;     // Zeeman shift / dlambdaD
  float a;      // damping
  // absorption-matrix coefficients (psi = 0 frame): with Hsum = H_b + H_r,
  // eta_I = 1 + c1 H_p + c2 Hsum, eta_L = c1 (H_p - Hsum/2) = c1 H_p - c3 Hsum,
  // eta_V = c4 (H_r - H_b), and the rho's likewise with F.
  float c1;     // eta0 sin^2(g) / 2
  float c2;     // eta0 (1 + cos^2 g) / 4
  float c3;     // eta0 sin^2(g) / 4
  float c4;     // eta0 cos(g) / 2
  // inclination derivatives (per degree): d eta_I/dg = d eta_L/dg =
  // g1 (H_p - Hsum/2), d eta_V/dg = g2 (H_r - H_b), rho's likewise
  float g1;     // eta0 sin(2g) / 2 * pi/180
  float g2;     // -eta0 sin(g) / 2 * pi/180
};

__device__ __forceinline__ PixK make_pixk(const LineK& lk, float B, float gam_deg,
                                          float eta0, float dld, float a, float v) {
  PixK P;
  P.invD = __frcp_rn(dld);
  P.uv = lk.cv * v * P.invD;
  P.uB = lk.cB * B * P.invD;
  P.a = a;
  float sg, cg;
  sincosf(gam_deg * kDeg, &sg, &cg);
  const float s2 = sg * sg;
  P.c1 = 0.5f * eta0 * s2;
  P.c2 = 0.25f * eta0 * fmaf(cg, cg, 1.0f);
  P.c3 = 0.25f * eta0 * s2;
  P.c4 = 0.5f * eta0 * cg;
  P.g1 = eta0 * sg * cg * kDeg;
  P.g2 = -0.5f * eta0 * sg * kDeg;
  return P;
}

// Per-pixel factors applied to the filtered derivative rows after the
// wavelength loop (they do not depend on wavelength): row r of the
// accumulators times rowscale[r] is d(unit-S1 Stokes)/d(parameter).
struct RowScale {
  float s[7];
};
__device__ __forceinline__ RowScale row_scale(const LineK& lk, float eta0, float dld) {
  RowScale R;
  const float invD = __frcp_rn(dld);
  R.s[0] = 1.0f;               // Stokes
  R.s[1] = lk.cB * invD;       // B: du_blue/dB = -du_red/dB
  R.s[2] = 1.0f;               // gamma (per degree)
  R.s[3] = __frcp_rn(eta0);    // eta0: the elements are linear in eta0
  R.s[4] = -invD;              // dlambdaD: du_k/d dlambdaD = -u_k / dlambdaD
  R.s[5] = 1.0f;               // damping
  R.s[6] = -lk.cv * invD;      // v: du_k/dv = -cv / dlambdaD
  return R;
}

// Accumulator layout of the fused pass: row r = 0 holds the unit-S1 Stokes
// profile K^{-1} e0 (I, Q0, U0, V in the psi = 0 frame); rows 1..6 hold
// (up to the row scales above) its derivatives with respect to B, gamma,
// eta0, dlambdaD, a, v_los.
constexpr int kRows = 7;
constexpr int kRowB = 1, kRowG = 2, kRowE = 3, kRowD = 4, kRowA = 5, kRowV = 6;

// One wavelength point: synthesis (and, if DERIV, the Jacobian rows),
// accumulated into acc[row][stokes][k] += T_k * value.
// Rows of the non-magnetic (B = 0) Stokes I profile used when the filling
// factor is free: value, then eta0 d/d eta0, u d/du, d/da, d/du (the scale
// factors of the magnetic rows E, D, A, V apply to them alike).
constexpr int kNmRows = 5;

template <int NF, bool DERIV, bool NM = false>
__device__ __forceinline__ void lambda_step(const Weideman& W, const PixK& P, float x,
                                            const float (&T)[NF],
                                            float (&acc)[DERIV ? kRows : 1][4][NF],
                                            float (*accn)[NF] = nullptr) {
  const float up = fmaf(x, P.invD, -P.uv);
  const float ub = up + P.uB, ur = up - P.uB;
  float Hp, Fp, Hb, Fb, Hr, Fr;
  faddeeva(W, up, P.a, Hp, Fp);
  faddeeva(W, ub, P.a, Hb, Fb);
  faddeeva(W, ur, P.a, Hr, Fr);
  const float Hsum = Hb + Hr, Hdif = Hr - Hb;
  const float Fsum = Fb + Fr, Fdif = Fr - Fb;
  // absorption-matrix elements (psi = 0 frame)
  // (linear-polarisation elements written as c1 (X_p - Xsum/2): exactly zero
  // when the three components coincide, B = 0)
  const float hL = fmaf(-0.5f, Hsum, Hp), fL = fmaf(-0.5f, Fsum, Fp);
  const float eI = fmaf(P.c1, Hp, fmaf(P.c2, Hsum, 1.0f));
  const float eL = P.c1 * hL;
  const float eV = P.c4 * Hdif;
  const float rL = P.c1 * fL;
  const float rV = P.c4 * Fdif;
  // closed-form Unno-Rachkovsky solution, unit S1, psi = 0 frame
  const float eI2 = eI * eI;
  const float Pi = fmaf(eL, rL, eV * rV);
  const float rr = fmaf(rL, rL, rV * rV);
  const float g = eI2 - fmaf(eL, eL, eV * eV) + rr;
  const float Dl = fmaf(eI2, g, -Pi * Pi);
  const float iD = rcp_fast(Dl);
  const float NI = eI * (eI2 + rr);
  const float NQ = fmaf(eI2, eL, rL * Pi);
  const float NU = eI * fmaf(eL, rV, -eV * rL);
  const float NV = fmaf(eI2, eV, rV * Pi);
  const float yI = NI * iD, yQ = -NQ * iD, yU = -NU * iD, yV = -NV * iD;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    acc[0][0][k] = fmaf(T[k], yI, acc[0][0][k]);
    acc[0][1][k] = fmaf(T[k], yQ, acc[0][1][k]);
    acc[0][2][k] = fmaf(T[k], yU, acc[0][2][k]);
    acc[0][3][k] = fmaf(T[k], yV, acc[0][3][k]);
  }
  if constexpr (DERIV) {
    // Eqs. 8-9: alpha = dH/da = -dF/du, beta = dH/du = dF/da
    const float a2 = 2.0f * P.a;
    const float alp = fmaf(a2, Hp, fmaf(2.0f * up, Fp, -kTwoInvSqrtPi));
    const float alb = fmaf(a2, Hb, fmaf(2.0f * ub, Fb, -kTwoInvSqrtPi));
    const float alr = fmaf(a2, Hr, fmaf(2.0f * ur, Fr, -kTwoInvSqrtPi));
    const float bep = fmaf(a2, Fp, -2.0f * up * Hp);
    const float beb = fmaf(a2, Fb, -2.0f * ub * Hb);
    const float ber = fmaf(a2, Fr, -2.0f * ur * Hr);
    // partials of Delta w.r.t. (eI, eL, eV, rL, rV)
    const float dDe = 2.0f * eI * (eI2 + g);
    const float dDq = -2.0f * NQ, dDv = -2.0f * NV;
    const float dDr = 2.0f * fmaf(eI2, rL, -Pi * eL);
    const float dDt = 2.0f * fmaf(eI2, rV, -Pi * eV);
    const float e2 = 2.0f * eI;
    // inclination derivatives of the elements
    const float gIL = P.g1 * hL;
    const float gV = P.g2 * Hdif;
    const float gRL = P.g1 * fL;
    const float gRV = P.g2 * Fdif;
#if VFISV_FOLD_ID_IN_WEIGHTS
    // Weights of the derivative rows: the 1/Delta of every partial is folded
    // into the filter weight.
    float Td[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) Td[k] = T[k] * iD;
#else
    const float (&Td)[NF] = T;
#endif

    // For each Stokes parameter: the partials p_X = Delta * dy_S/dX w.r.t.
    // the five elements, then the chain rule through the profiles.
    auto stokes = [&](int S, float pe, float pq, float pv, float pr, float pt) {
      // d/dH_k and d/dF_k of the component profiles
      const float peq = pe + pq;
      const float SHp = peq * P.c1;
      const float tH = fmaf(pe, P.c2, -pq * P.c3);
      const float SHb = fmaf(-pv, P.c4, tH), SHr = fmaf(pv, P.c4, tH);
      const float SFp = pr * P.c1;
      const float tF = -pr * P.c3;
      const float SFb = fmaf(-pt, P.c4, tF), SFr = fmaf(pt, P.c4, tF);
      // d/du_k = dS/dH beta - dS/dF alpha
      const float Gp = fmaf(SHp, bep, -SFp * alp);
      const float Gb = fmaf(SHb, beb, -SFb * alb);
      const float Gr = fmaf(SHr, ber, -SFr * alr);
      float vB = Gb - Gr;                                  // x kB
      float vG = fmaf(peq, gIL, fmaf(pv, gV, fmaf(pr, gRL, pt * gRV)));
      float vE = fmaf(pe, eI - 1.0f, fmaf(pq, eL, fmaf(pv, eV, fmaf(pr, rL, pt * rV))));
      float vD = fmaf(up, Gp, fmaf(ub, Gb, ur * Gr));      // x (-1/dlambdaD)
      float vA = fmaf(SHp, alp, fmaf(SFp, bep, fmaf(SHb, alb, fmaf(SFb, beb,
                       fmaf(SHr, alr, SFr * ber)))));
      float vV = Gp + Gb + Gr;                             // x kv
#if !VFISV_FOLD_ID_IN_WEIGHTS
      // the 1/Delta of every partial, applied to the six row values
      vB *= iD; vG *= iD; vE *= iD; vD *= iD; vA *= iD; vV *= iD;
#endif
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        acc[kRowB][S][k] = fmaf(Td[k], vB, acc[kRowB][S][k]);
        acc[kRowG][S][k] = fmaf(Td[k], vG, acc[kRowG][S][k]);
        acc[kRowE][S][k] = fmaf(Td[k], vE, acc[kRowE][S][k]);
        acc[kRowD][S][k] = fmaf(Td[k], vD, acc[kRowD][S][k]);
        acc[kRowA][S][k] = fmaf(Td[k], vA, acc[kRowA][S][k]);
        acc[kRowV][S][k] = fmaf(Td[k], vV, acc[kRowV][S][k]);
      }
    };
    // y_S = s N_S / Delta => Delta dy_S/dX = s dN_S/dX - y_S dDelta/dX
    stokes(0, fmaf(-yI, dDe, fmaf(3.0f, eI2, rr)), -yI * dDq, -yI * dDv,
           fmaf(-yI, dDr, e2 * rL), fmaf(-yI, dDt, e2 * rV));
    stokes(1, fmaf(-yQ, dDe, -e2 * eL), fmaf(-yQ, dDq, -fmaf(rL, rL, eI2)),
           fmaf(-yQ, dDv, -rL * rV), fmaf(-yQ, dDr, -fmaf(rL, eL, Pi)),
           fmaf(-yQ, dDt, -rL * eV));
    stokes(2, fmaf(-yU, dDe, -fmaf(eL, rV, -eV * rL)), fmaf(-yU, dDq, -eI * rV),
           fmaf(-yU, dDv, eI * rL), fmaf(-yU, dDr, eI * eV), fmaf(-yU, dDt, -eI * eL));
    stokes(3, fmaf(-yV, dDe, -e2 * eV), fmaf(-yV, dDq, -rV * rL),
           fmaf(-yV, dDv, -fmaf(rV, rV, eI2)), fmaf(-yV, dDr, -rV * eL),
           fmaf(-yV, dDt, -fmaf(rV, eV, Pi)));
    if constexpr (NM) {
      // B = 0: the three components coincide with the pi one, eta_I =
      // 1 + eta0 H_p, no polarisation, I = 1 / eta_I (unit S1)
      const float eta0 = fmaf(2.0f, P.c2, P.c1);
      const float yn = rcp_fast(fmaf(eta0, Hp, 1.0f));
      const float ny2 = -eta0 * yn * yn;
      const float nU = ny2 * bep;  // d/du_p
      const float nv[kNmRows] = {yn, ny2 * Hp, up * nU, ny2 * alp, nU};
#pragma unroll
      for (int k = 0; k < NF; ++k)
#pragma unroll
        for (int r = 0; r < kNmRows; ++r) accn[r][k] = fmaf(T[k], nv[r], accn[r][k]);
    }
  }
}

}  // namespace vfisv
