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
// passes over the observables (J^T W r and the first rows of J^T W J, then
// the rest), half of them live at a time; the second pass runs where
// `second` holds and recomputes the Jacobian rows.  The observables run in
// a runtime loop so the block stays small in the instruction cache.
template <int NF, int NP, bool AF, bool SPLIT, class Fetch>
__device__ __forceinline__ void build_normal_equations(
    Fetch& fetch, const float* __restrict__ tau, float* __restrict__ scr, int64_t ns, float mus1, float c2p,
    float s2p, float s0, float alf, float mu, const RowScale& R, bool keepA, bool store,
    bool second) {
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
  // J^T W J entries of pass 0 (all of them without the split: pass 2)
  constexpr int kSplit = SPLIT ? (NPK + NP) / 2 - NP : NPK;
  auto build = [&](auto half) {
    constexpr int H = decltype(half)::value;
    constexpr int NA = (H == 1) ? NPK - kSplit : NP + kSplit;
    Dot2 acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = Dot2{0.0f, 0.0f};
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
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float wj = ww * J[p];
        if constexpr (H != 1) acc[p].add(wj, rr);
#pragma unroll
        for (int q = 0; q <= p; ++q) {
          const int e = tri(p, q);
          if (H != 1 && e < kSplit && !keepA) acc[NP + e].add(wj, J[q]);
          if (H == 1 && e >= kSplit) acc[e - kSplit].add(wj, J[q]);
        }
      }
    }
    if constexpr (H != 1) {
      if (store) {
#pragma unroll
        for (int i = 0; i < NP; ++i) scr[(int64_t)(NPK + i) * ns] = acc[i].value();
        if (!keepA) {
#pragma unroll
          for (int e = 0; e < kSplit; ++e) scr[(int64_t)e * ns] = acc[NP + e].value();
        }
      }
    } else {
      if (store && !keepA) {
#pragma unroll
        for (int e = kSplit; e < NPK; ++e) scr[(int64_t)e * ns] = acc[e - kSplit].value();
      }
    }
  };
  if constexpr (SPLIT) {
    build(Half<0>{});
    if (second) build(Half<1>{});
  } else {
    build(Half<2>{});
  }
}

}  // namespace vfisv
