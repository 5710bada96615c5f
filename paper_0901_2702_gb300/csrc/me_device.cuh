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
#pragma unroll
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

// Per-pixel constants of one synthesis.
struct PixK {
  float invD;   // 1 / dlambdaD
  float uv;     // Doppler shift / dlambdaD
  float uB;     // Zeeman shift / dlambdaD
  float a;      // damping
  float eta0;
  float s2;     // sin^2 gamma
  float c2p1;   // 1 + cos^2 gamma
  float cg;     // cos gamma
  // derivative helpers
  float kB;     // d u_blue / dB = cB / dlambdaD
  float kv;     // d u / dv = -cv / dlambdaD
  float ds2;    // d sin^2 gamma / d gamma[deg]
  float dcg;    // d cos gamma / d gamma[deg]
};

__device__ __forceinline__ PixK make_pixk(const LineK& lk, float B, float gam_deg,
                                          float eta0, float dld, float a, float v) {
  PixK P;
  P.invD = __frcp_rn(dld);
  P.uv = lk.cv * v * P.invD;
  P.uB = lk.cB * B * P.invD;
  P.a = a;
  P.eta0 = eta0;
  float sg, cg;
  sincosf(gam_deg * kDeg, &sg, &cg);
  P.s2 = sg * sg;
  P.c2p1 = fmaf(cg, cg, 1.0f);
  P.cg = cg;
  P.kB = lk.cB * P.invD;
  P.kv = -lk.cv * P.invD;
  P.ds2 = 2.0f * sg * cg * kDeg;
  P.dcg = -sg * kDeg;
  return P;
}

// Accumulator layout of the fused pass: row r = 0 holds the unit-S1 Stokes
// profile K^{-1} e0 (I, Q0, U0, V in the psi = 0 frame); rows 1..6 hold its
// derivatives with respect to B, gamma, eta0, dlambdaD, a, v_los.
constexpr int kRows = 7;
constexpr int kRowB = 1, kRowG = 2, kRowE = 3, kRowD = 4, kRowA = 5, kRowV = 6;

// One wavelength point: synthesis (and, if DERIV, the Jacobian rows),
// accumulated into acc[row][stokes][k] += T_k * value.
template <int NF, bool DERIV>
__device__ __forceinline__ void lambda_step(const Weideman& W, const PixK& P, float x,
                                            const float (&T)[NF],
                                            float (&acc)[DERIV ? kRows : 1][4][NF]) {
  const float up = fmaf(x, P.invD, -P.uv);
  const float ub = up + P.uB, ur = up - P.uB;
  float Hp, Fp, Hb, Fb, Hr, Fr;
  faddeeva(W, up, P.a, Hp, Fp);
  faddeeva(W, ub, P.a, Hb, Fb);
  faddeeva(W, ur, P.a, Hr, Fr);
  const float Hs = 0.5f * (Hb + Hr), Hd = 0.5f * (Hr - Hb);
  const float Fs = 0.5f * (Fb + Fr), Fd = 0.5f * (Fr - Fb);
  // absorption-matrix elements per unit eta0 (psi = 0 frame)
  const float uI = 0.5f * fmaf(Hp, P.s2, Hs * P.c2p1);
  const float uL = 0.5f * (Hp - Hs) * P.s2;
  const float uV = Hd * P.cg;
  const float urL = 0.5f * (Fp - Fs) * P.s2;
  const float urV = Fd * P.cg;
  const float eI = fmaf(P.eta0, uI, 1.0f);
  const float eL = P.eta0 * uL, eV = P.eta0 * uV;
  const float rL = P.eta0 * urL, rV = P.eta0 * urV;
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
    // partials of Delta and of the numerators w.r.t. (eI, eL, eV, rL, rV)
    const float dDe = 2.0f * eI * (eI2 + g);
    const float dDq = -2.0f * NQ, dDv = -2.0f * NV;
    const float dDr = 2.0f * fmaf(eI2, rL, -Pi * eL);
    const float dDt = 2.0f * fmaf(eI2, rV, -Pi * eV);
    // y_S = s N_S / Delta  =>  dy_S/dX = (s dN_S/dX - y_S dDelta/dX) / Delta
    const float Ie = iD * (fmaf(3.0f, eI2, rr) - yI * dDe);
    const float Iq = -iD * yI * dDq, Iv = -iD * yI * dDv;
    const float Ir = iD * (2.0f * eI * rL - yI * dDr);
    const float It = iD * (2.0f * eI * rV - yI * dDt);
    const float Qe = -iD * (2.0f * eI * eL + yQ * dDe);
    const float Qq = -iD * (fmaf(rL, rL, eI2) + yQ * dDq);
    const float Qv = -iD * (rL * rV + yQ * dDv);
    const float Qr = -iD * (fmaf(rL, eL, Pi) + yQ * dDr);
    const float Qt = -iD * (rL * eV + yQ * dDt);
    const float Ue = -iD * (fmaf(eL, rV, -eV * rL) + yU * dDe);
    const float Uq = -iD * (eI * rV + yU * dDq);
    const float Uv = -iD * (-eI * rL + yU * dDv);
    const float Ur = -iD * (-eI * eV + yU * dDr);
    const float Ut = -iD * (eI * eL + yU * dDt);
    const float Ve = -iD * (2.0f * eI * eV + yV * dDe);
    const float Vq = -iD * (rV * rL + yV * dDq);
    const float Vv = -iD * (fmaf(rV, rV, eI2) + yV * dDv);
    const float Vr = -iD * (rV * eL + yV * dDr);
    const float Vt = -iD * (fmaf(rV, eV, Pi) + yV * dDt);

    auto push = [&](int row, float de, float dq, float dv, float dr, float dt) {
      const float dI = fmaf(Ie, de, fmaf(Iq, dq, fmaf(Iv, dv, fmaf(Ir, dr, It * dt))));
      const float dQ = fmaf(Qe, de, fmaf(Qq, dq, fmaf(Qv, dv, fmaf(Qr, dr, Qt * dt))));
      const float dU = fmaf(Ue, de, fmaf(Uq, dq, fmaf(Uv, dv, fmaf(Ur, dr, Ut * dt))));
      const float dV = fmaf(Ve, de, fmaf(Vq, dq, fmaf(Vv, dv, fmaf(Vr, dr, Vt * dt))));
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        acc[row][0][k] = fmaf(T[k], dI, acc[row][0][k]);
        acc[row][1][k] = fmaf(T[k], dQ, acc[row][1][k]);
        acc[row][2][k] = fmaf(T[k], dU, acc[row][2][k]);
        acc[row][3][k] = fmaf(T[k], dV, acc[row][3][k]);
      }
    };
    // element derivatives from profile derivatives (pi, sigma sum, sigma difference)
    auto shape = [&](int row, float dHp, float dHs, float dHd, float dFp, float dFs, float dFd) {
      const float e = P.eta0;
      push(row, e * 0.5f * fmaf(dHp, P.s2, dHs * P.c2p1), e * 0.5f * (dHp - dHs) * P.s2,
           e * dHd * P.cg, e * 0.5f * (dFp - dFs) * P.s2, e * dFd * P.cg);
    };
    // B: only the sigma components move, u_b = u_p + uB, u_r = u_p - uB
    {
      const float h = 0.5f * P.kB;
      shape(kRowB, 0.0f, h * (beb - ber), -h * (beb + ber), 0.0f, h * (alr - alb), h * (alb + alr));
    }
    // gamma (per degree)
    {
      const float he = 0.5f * P.eta0;
      const float dIL = he * (Hp - Hs) * P.ds2;
      push(kRowG, dIL, dIL, P.eta0 * Hd * P.dcg, he * (Fp - Fs) * P.ds2, P.eta0 * Fd * P.dcg);
    }
    // eta0: the elements are linear in it
    push(kRowE, uI, uL, uV, urL, urV);
    // dlambdaD: d u_k / d dlambdaD = -u_k / dlambdaD
    {
      const float ip = up * P.invD, ib = ub * P.invD, ir = ur * P.invD;
      const float hbp = -bep * ip, hbb = -beb * ib, hbr = -ber * ir;
      const float fap = alp * ip, fab = alb * ib, far_ = alr * ir;
      shape(kRowD, hbp, 0.5f * (hbb + hbr), 0.5f * (hbr - hbb), fap, 0.5f * (fab + far_),
            0.5f * (far_ - fab));
    }
    // damping: dH/da = alpha, dF/da = beta
    shape(kRowA, alp, 0.5f * (alb + alr), 0.5f * (alr - alb), bep, 0.5f * (beb + ber),
          0.5f * (ber - beb));
    // v_los: d u_k / dv = kv for all components
    {
      const float kv = P.kv;
      shape(kRowV, kv * bep, kv * 0.5f * (beb + ber), kv * 0.5f * (ber - beb), -kv * alp,
            -kv * 0.5f * (alb + alr), -kv * 0.5f * (alr - alb));
    }
  }
}

}  // namespace vfisv
