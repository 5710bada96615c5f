// Device pieces shared by the Levenberg-Marquardt kernels (invert.cu,
// invert_ws.cu): the compensated dot product and the build of J^T W J and
// J^T W r at an accepted model (Eqs. 3-4) from the filtered rows of a pass.
#pragma once

#include "solve.cuh"

namespace vfisv {

// Compensated accumulation of a product: s + c tracks sum(a*b) to about
// twice the working precision (TwoProduct via FMA, TwoSum).
struct Dot2 {
  float s, c;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float ep = fmaf(a, b, -p);
    const float t = s + p;
    const float bp = t - s;
    const float es = (s - (t - bp)) + (p - bp);
    s = t;
    c += es + ep;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

// Two compensated sums advanced together by the packed FP32x2 instructions
// of sm_100 and later: each lane performs exactly Dot2::add's IEEE
// operations (the error term is carried negated: fma(-a, b, p) is
// -(a b - p) with the same single rounding, and c - (-e) is c + e).
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
        "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&r);
}

struct Dot2x2 {
  float2 s, c;
  __device__ __forceinline__ void add(float2 a, float2 na, float2 b) {
    const float2 p = __fmul2_rn(a, b);
    const float2 e = __ffma2_rn(na, b, p);  // -(a b - p)
    const float2 t = __fadd2_rn(s, p);
    const float2 bp = fsub2(t, s);
    const float2 es = __fadd2_rn(fsub2(s, fsub2(t, bp)), fsub2(p, bp));
    s = t;
    c = __fadd2_rn(c, fsub2(es, e));
  }
};

// Compile-time index of a pass (template argument of a generic lambda).
template <int H>
struct Half {
  static constexpr int value = H;
};

// The filtered rows one observable (Stokes s of filter k) needs: the seven
// rows (unit-S1 Stokes, then the derivative rows of B, gamma, eta0,
// dlambdaD, a, v) at the two psi = 0 frame Stokes it is built from (sa, sb:
// I, I for s = 0; Q0, U0 for s = 1, 2; V, V for s = 3), and, with the
// filling factor free, the non-magnetic rows of filter k.
struct ObsRows {
  float a[kRows], b[kRows];
  float n[kNmRows];
  float obs, w;  // the observed value and its weight
};

// Observed value and weight of observable (s, k) of a pixel (row-major
// [4][NF] rows o and wv), read by a row source's issue() with the rows.
template <int NF>
struct ObsRead {
  float o, w;
  __device__ __forceinline__ void issue(const float* __restrict__ obs,
                                        const float* __restrict__ wv, int k, int s) {
    o = obs[s * NF + k];
    w = wv[s * NF + k];
  }
};

__device__ __forceinline__ int obs_sa(int s) { return (s == 0) ? 0 : (s == 3 ? 3 : 1); }
__device__ __forceinline__ int obs_sb(int s) { return (s == 0) ? 0 : (s == 3 ? 3 : 2); }

// J^T W J (packed lower triangle, e < NPK) and J^T W r (after it) of the
// 4 NF observables in compensated FP32 sums, written to scr[e * ns] where
// `store` holds (J^T W J only without keepA).  The filtered rows come from
// `fetch`: fetch.issue(k, s) starts reading the rows of observable (Stokes
// s, filter k) with its observed value and weight, and fetch.take(k, s,
// rows) completes that read; the next
// observable's read is issued before the current one is summed, so a
// source with latency (tensor memory) overlaps the arithmetic.  psi, S0
// and S1 enter after filtering.  With SPLIT the sums are built in two
// passes over the observables (the first parameter rows, then the rest),
// half of them live at a time; the second pass recomputes the Jacobian
// rows.  The observables run in a runtime loop so the block stays small in
// the instruction cache.
template <int NF, int NP, bool AF, bool SPLIT, class Fetch>
__device__ __forceinline__ void build_normal_equations(
    Fetch& fetch, const float* __restrict__ tau, float* __restrict__ scr, int64_t ns, float mus1, float c2p,
    float s2p, float s0, float alf, float mu, const RowScale& R, bool keepA, bool store) {
  constexpr int NPK = NP * (NP + 1) / 2;
  // Jacobian row and residual of observable (s, k): row r gives
  // fmaf(cA, a[r], cB * b[r]), the psi rotation of Q0/U0.
  auto jac = [&](int k, int s, const ObsRows& rows, float (&J)[NP], float& rr, float& ww) {
    constexpr int rowOf[10] = {kRowB, kRowG, -1, kRowE, kRowD, kRowA, kRowV, -1, -1, -1};
    // rows of the non-magnetic profile for eta0, dlambdaD, a, v (AF)
    constexpr int nmRowOf[10] = {-1, -1, -1, 1, 2, 3, 4, -1, -1, -1};
    const float cA = (s == 1) ? c2p : (s == 2 ? s2p : 1.0f);
    const float cB = (s == 1) ? -s2p : (s == 2 ? c2p : 0.0f);
#pragma unroll
    for (int p = 0; p < NP; ++p)
      if (rowOf[p] >= 0) {
        J[p] = (alf * mus1 * R.s[rowOf[p]]) * fmaf(cA, rows.a[rowOf[p]], cB * rows.b[rowOf[p]]);
        if (AF && nmRowOf[p] > 0 && s == 0)
          J[p] = fmaf((1.0f - alf) * mus1 * R.s[rowOf[p]], rows.n[nmRowOf[p]], J[p]);
      }
    J[2] = 0.0f;  // psi only rotates Q and U
    if (s == 1 || s == 2) {
      const float q0 = alf * rows.a[0], u0 = alf * rows.b[0];
      const float Qk = mus1 * fmaf(c2p, q0, -s2p * u0);
      const float Uk = mus1 * fmaf(s2p, q0, c2p * u0);
      J[2] = (s == 1) ? -2.0f * kDeg * Uk : 2.0f * kDeg * Qk;
    }
    J[7] = (s == 0) ? tau[k] : 0.0f;
    const float linm = fmaf(cA, rows.a[0], cB * rows.b[0]);  // magnetic
    const float lin =
        AF ? ((s == 0) ? fmaf(alf, linm - rows.n[0], rows.n[0]) : alf * linm) : linm;
    J[8] = mu * lin;
    if constexpr (AF) J[NP - 1] = mus1 * ((s == 0) ? linm - rows.n[0] : linm);
    const float sv = (s == 0) ? fmaf(s0, tau[k], mus1 * lin) : mus1 * lin;
    ww = rows.w;
    rr = rows.obs - sv;
  };
  // The sums of parameter row p are J^T W r_p and J^T W J_pq, q <= p: all
  // take the product with w J_p, so they are advanced in pairs by packed
  // instructions: (J^T W r_p, J^T W J_p0), (J^T W J_p1, J^T W J_p2), ...,
  // the last pair of an odd row holding a lane that is not stored.  With
  // SPLIT, pass 0 takes rows 0 .. PS - 1 and pass 1 the others (27 sums
  // each for 9 parameters); otherwise one pass takes every row.
  constexpr int NB = (NP + 2) / 2;                  // pairs of (r, J_0, ..., J_{NP-1})
  constexpr int PS = SPLIT ? (NP == 9 ? 6 : NP) : NP;
  auto pairs = [](int p) { return (p + 3) / 2; };  // pairs of row p
  auto build = [&](auto half) {
    constexpr int H = decltype(half)::value;
    constexpr int P0 = (H == 1) ? PS : 0, P1 = (H == 0 && SPLIT) ? PS : NP;
    constexpr int NS = [] {
      int n = 0;
      for (int p = P0; p < P1; ++p) n += (p + 3) / 2;
      return n;
    }();
    Dot2x2 acc[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) acc[i] = Dot2x2{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    // observables filter-major (k outer, s inner)
    fetch.issue(0, 0);
#pragma unroll 1
    for (int i = 0; i < 4 * NF; ++i) {
      const int k = i >> 2, s = i & 3;
      ObsRows rows;
      fetch.take(k, s, rows);
      if (i + 1 < 4 * NF) fetch.issue((i + 1) >> 2, (i + 1) & 3);
      float J[NP], rr, ww;
      jac(k, s, rows, J, rr, ww);
      // (r, J_0), (J_1, J_2), ...; a lane past J_{NP-1} is zero
      float2 bq[NB];
#pragma unroll
      for (int m = 0; m < NB; ++m)
        bq[m] = make_float2(m == 0 ? rr : J[2 * m - 1], (2 * m < NP) ? J[2 * m] : 0.0f);
      int base = 0;
#pragma unroll
      for (int p = P0; p < P1; ++p) {
        const float wj = ww * J[p];
        const float2 a = make_float2(wj, wj), na = make_float2(-wj, -wj);
#pragma unroll
        for (int m = 0; m < pairs(p); ++m) acc[base + m].add(a, na, bq[m]);
        base += pairs(p);
      }
    }
    if (store) {
      int base = 0;
#pragma unroll
      for (int p = P0; p < P1; ++p) {
#pragma unroll
        for (int m = 0; m < pairs(p); ++m) {
          const Dot2x2& d = acc[base + m];
          // lane x: J^T W r_p (m = 0) or J^T W J_p,2m-1; lane y: J^T W J_p,2m
          const float vx = d.s.x + d.c.x, vy = d.s.y + d.c.y;
          if (m == 0)
            scr[(int64_t)(NPK + p) * ns] = vx;
          else if (!keepA)
            scr[(int64_t)tri(p, 2 * m - 1) * ns] = vx;
          if (2 * m <= p && !keepA) scr[(int64_t)tri(p, 2 * m) * ns] = vy;
        }
        base += pairs(p);
      }
    }
  };
  if constexpr (SPLIT) {
    build(Half<0>{});
    build(Half<1>{});
  } else {
    build(Half<2>{});
  }
}

}  // namespace vfisv
