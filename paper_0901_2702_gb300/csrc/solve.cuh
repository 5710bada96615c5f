// The FP64 pieces of the damped Levenberg-Marquardt solve (Eqs. 3-6) and of
// the covariance, shared by the LM kernels: Table 2's damping rule, the
// Jacobi-scaled normal equations, Cholesky with a Jacobi-eigenvalue (SVD)
// fallback.  The normal equations are read as packed floats at
// scr[e * ns], e = 0..44 the lower triangle of J^T W J, 45..53 J^T W r.
#pragma once

#include <math.h>

#include "common.cuh"

namespace vfisv {

constexpr int kNP = 9;    // parameters taking part in the solve (alpha held)
constexpr int kNPk = 45;  // packed lower triangle of a 9x9 matrix
// With the filling factor free the solve takes N = 10 parameters; the
// functions below are templates on N (default 9).

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

// 2^e as a float / double built from its exponent bits (e clamped to the
// normal range); a product with it is exact unless the result leaves the
// normal range.
__device__ __forceinline__ float pow2f(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((e + 127) << 23);
}
__device__ __forceinline__ double pow2d(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// Table 2 (with the oracle's reading of its overlapping rows).
__device__ __forceinline__ double eps_update(double e, bool success) {
  double n;
  if (success)
    n = (e > 1e4) ? e / 100.0 : (e >= 1e-4 ? e / 10.0 : e / 2.0);
  else
    n = (e < 1e-4) ? e * 100.0 : (e <= 1e4 ? e * 2.0 : e * 10.0);
  return fmax(n, 1e-9);  // floor: the scaled damped matrix keeps eigenvalues >= 1e-9
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations, FP64; the
// fallback when the Cholesky pivots show a (numerically) singular matrix.
// Solves M y = b with eigenvalues below 1e-12 * max zeroed (truncated SVD
// of a symmetric matrix), or, with b == nullptr, writes the truncated
// pseudo-inverse into Minv.
template <int N = kNP>
static __device__ __noinline__ void jacobi_pinv(const double* Mp /*packed*/, const double* b,
                                         double* y, double* Minv) {
  double a[N][N], v[N][N];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      a[i][j] = (i >= j) ? Mp[tri(i, j)] : Mp[tri(j, i)];
      v[i][j] = (i == j) ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = 0; i < N; ++i) {
      dia += a[i][i] * a[i][i];
      for (int j = i + 1; j < N; ++j) off += a[i][j] * a[i][j];
    }
    if (!(off > 1e-26 * dia)) break;  // off-diagonal below ~3e-13 of the diagonal
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        const double apq = a[p][q];
        if (apq == 0.0) continue;
        const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < N; ++k) {
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < N; ++k) {
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < N; ++k) {
          const double vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
  double lmax = 0.0;
  for (int i = 0; i < N; ++i) lmax = fmax(lmax, fabs(a[i][i]));
  double linv[N];
  for (int i = 0; i < N; ++i) {
    const double l = fabs(a[i][i]);
    linv[i] = (l > 1e-12 * lmax && l > 0.0) ? 1.0 / a[i][i] : 0.0;
  }
  if (b) {
    double t[N];
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
      for (int k = 0; k < N; ++k) s += v[k][i] * b[k];
      t[i] = s * linv[i];
    }
    for (int k = 0; k < N; ++k) {
      double s = 0.0;
      for (int i = 0; i < N; ++i) s += v[k][i] * t[i];
      y[k] = s;
    }
  } else {
    for (int i = 0; i < N; ++i)
      for (int j = 0; j <= i; ++j) {
        double s = 0.0;
        for (int k = 0; k < N; ++k) s += v[i][k] * linv[k] * v[j][k];
        Minv[tri(i, j)] = s;
      }
  }
}

// In-place Cholesky of a packed 9x9 matrix; false if a pivot is not
// comfortably positive (the matrix has unit-scale diagonal here).  The
// diagonal receives the reciprocal pivots 1 / L_jj, which is all the
// substitutions and the inverse use of it (one array fewer in registers).
template <int N = kNP>
__device__ __forceinline__ bool cholesky9(double (&L)[(N * (N + 1) / 2)]) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    double d = L[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; ++k) d = fma(-L[tri(j, k)], L[tri(j, k)], d);
    if (!(d > 1e-10)) return false;
    const double r = rsqrt(d);
    L[tri(j, j)] = r;
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      double s = L[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) s = fma(-L[tri(i, k)], L[tri(j, k)], s);
      L[tri(i, j)] = s * r;
    }
  }
  return true;
}

// Forward and back substitution with the factor (reciprocal pivots on its
// diagonal).
template <int N = kNP>
__device__ __forceinline__ void chol_solve9(const double (&L)[(N * (N + 1) / 2)], double (&x)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = x[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = fma(-L[tri(i, k)], x[k], s);
    x[i] = s * L[tri(i, i)];
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    double s = x[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) s = fma(-L[tri(k, i)], x[k], s);
    x[i] = s * L[tri(i, i)];
  }
}

// In place, from the Cholesky factor L (reciprocal pivots on its diagonal) of M: first
// the triangular inverse W = L^-1 (columns right to left, each from the
// already inverted trailing block), then M^-1 = W^T W (columns left to
// right: entry (i, j) needs only rows >= i of columns j and i, which are
// still W) -- ~285 FMAs against ~810 for N solves with unit vectors.
template <int N = kNP>
__device__ __forceinline__ void chol_inverse(double (&L)[(N * (N + 1) / 2)]) {
#pragma unroll
  for (int j = N - 1; j >= 0; --j) {
    // W[i][j] = -ri[j] * sum_{k=j+1..i} W[i][k] L[k][j]   (i > j)
#pragma unroll
    for (int i = N - 1; i > j; --i) {
      double s = 0.0;
#pragma unroll
      for (int k = j + 1; k <= i; ++k) s = fma(L[tri(i, k)], L[tri(k, j)], s);
      L[tri(i, j)] = -s * L[tri(j, j)];
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int i = j; i < N; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = i; k < N; ++k) s = fma(L[tri(k, i)], L[tri(k, j)], s);
      L[tri(i, j)] = s;
    }
}

// Jacobi-scaled matrix of the stored normal equations: returns the scale
// s_i = diag^-1/2 (0 for held parameters) and fills Mx = D^-1/2 A D^-1/2 +
// eps I on free parameters, identity rows/columns on held ones.
template <int N = kNP>
__device__ __forceinline__ void scaled_system(const float* scr, int64_t ns, uint32_t free_mask,
                                              double eps, double (&Mx)[(N * (N + 1) / 2)],
                                              double (&sc)[N], bool (&held)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const double d = (double)scr[(int64_t)tri(i, i) * ns];
    held[i] = !((free_mask >> i) & 1u) || !(d > 0.0) || !isfinite(d);
    sc[i] = held[i] ? 0.0 : rsqrt(d);
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      double m;
      if (i == j)
        m = held[i] ? 1.0 : 1.0 + eps;
      else
        m = (held[i] || held[j]) ? 0.0 : (double)scr[(int64_t)tri(i, j) * ns] * sc[i] * sc[j];
      Mx[tri(i, j)] = m;
    }
}

// Eq. 5 with the Marquardt diagonal (Eq. 4): delta = (A + eps diag A)^-1 g,
// in FP64 (the default precision of the solve).
//
// The system is balanced by a diagonal scaling P of powers of two before the
// factorisation: with A' = P A P (diagonal in [1/4, 1)), (A' + eps diag A') y
// = P g has the solution y = P^-1 delta, the same system.  Scaling by powers
// of two is exact (an exponent change in FP32, before the conversion to
// FP64), so the FP64 work is only the damped diagonal, the Cholesky
// factorisation and the substitutions; the rare fallback (a pivot below
// 1e-10) takes the unit-diagonal Jacobi scaling and the truncated
// eigen-decomposition.
// LEAN: the scaling exponents are read again from scr for the last step
// instead of staying live through the factorisation (for callers short of
// registers; scr must not change meanwhile).
template <int N = kNP, bool LEAN = false>
__device__ __forceinline__ void damped_step_fp64_body(const float* scr, int64_t ns,
                                                      uint32_t free_mask, double eps,
                                                      double (&delta)[N]) {
  double L[(N * (N + 1) / 2)];
  int ex[N];         // P_ii = 2^-ex[i]
  uint32_t hm = 0;   // bit i: parameter i held
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const float d = scr[(int64_t)tri(i, i) * ns];
    const bool h = !((free_mask >> i) & 1u) || !(d > 0.0f) || !isfinite(d);
    hm |= (h ? 1u : 0u) << i;
    int k = 0;
    frexpf(h ? 1.0f : d, &k);  // d = m 2^k, m in [1/2, 1)
    ex[i] = (k + 1) >> 1;      // d 2^-2ex in [1/4, 1)
  }
  const double one_eps = 1.0 + eps;
  float pw[N];
#pragma unroll
  for (int i = 0; i < N; ++i) pw[i] = pow2f(-ex[i]);
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const bool hi = (hm >> i) & 1u, hj = (hm >> j) & 1u;
      double m;
      if (i == j)
        m = hi ? 1.0 : (double)(scr[(int64_t)tri(i, i) * ns] * pw[i] * pw[i]) * one_eps;
      else
        m = (hi || hj) ? 0.0 : (double)(scr[(int64_t)tri(i, j) * ns] * pw[i] * pw[j]);
      L[tri(i, j)] = m;
    }
  double y[N];
#pragma unroll
  for (int i = 0; i < N; ++i)
    y[i] = ((hm >> i) & 1u) ? 0.0 : (double)(scr[(int64_t)((N * (N + 1) / 2) + i) * ns] * pw[i]);
  if (cholesky9<N>(L)) {
    chol_solve9<N>(L, y);
    if constexpr (LEAN) {
      asm volatile("" ::: "memory");  // read the diagonal again (no register kept)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        int k = 0;
        frexpf(((hm >> i) & 1u) ? 1.0f : scr[(int64_t)tri(i, i) * ns], &k);
        ex[i] = (k + 1) >> 1;
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) delta[i] = ((hm >> i) & 1u) ? 0.0 : y[i] * pow2d(-ex[i]);
    return;
  }
  // numerically singular: unit-diagonal Jacobi scaling, truncated
  // eigen-decomposition
  double sc[N], bv[N];
  bool held[N];
  scaled_system<N>(scr, ns, free_mask, eps, L, sc, held);
#pragma unroll
  for (int i = 0; i < N; ++i)
    bv[i] = held[i] ? 0.0 : (double)scr[(int64_t)((N * (N + 1) / 2) + i) * ns] * sc[i];
  jacobi_pinv<N>(L, bv, y, nullptr);
#pragma unroll
  for (int i = 0; i < N; ++i) delta[i] = held[i] ? 0.0 : sc[i] * y[i];
}

// The same step kept out of line (the LM kernel that calls it from the
// middle of its iteration gives it the whole register file).
template <int N = kNP>
static __device__ __noinline__ void damped_step_fp64(const float* scr, int64_t ns,
                                                     uint32_t free_mask, double eps,
                                                     double (&delta)[N]) {
  damped_step_fp64_body<N>(scr, ns, free_mask, eps, delta);
}

// Covariance (J^T W J)^+ at the final model, in parameter units, from the
// packed J^T W J at scr[e * ns].  Reads everything before writing `out`, so
// `out` may hold the packed matrix itself.  With try_only, returns false
// without writing when the Cholesky factorisation fails (the caller then
// runs the eigen-decomposition path for that pixel).
template <int N = kNP>
static __device__ __noinline__ bool covariance_fp64(const float* scr, int64_t ns, uint32_t free_mask,
                                        float* out, bool try_only) {
  double L[(N * (N + 1) / 2)], sc[N];
  bool held[N];
  scaled_system<N>(scr, ns, free_mask, 0.0, L, sc, held);
  if (cholesky9<N>(L)) {
    chol_inverse<N>(L);  // L now holds the scaled inverse
  } else {
    if (try_only) return false;
    double P[(N * (N + 1) / 2)];
    scaled_system<N>(scr, ns, free_mask, 0.0, L, sc, held);
    jacobi_pinv<N>(L, nullptr, nullptr, P);
#pragma unroll
    for (int e = 0; e < (N * (N + 1) / 2); ++e) L[e] = P[e];
  }
  // unscale each distinct entry once; rows are written as float pairs (a
  // row is 40 bytes, so 8-byte aligned when `out` is)
  float q[(N * (N + 1) / 2)];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j)
      q[tri(i, j)] = (held[i] || held[j]) ? 0.0f : (float)(sc[i] * sc[j] * L[tri(i, j)]);
  auto at = [&](int i, int j) -> float {
    return (i < N && j < N) ? q[i >= j ? tri(i, j) : tri(j, i)] : 0.0f;
  };
  if ((reinterpret_cast<uintptr_t>(out) & 7u) == 0) {
    float2* o2 = reinterpret_cast<float2*>(out);
#pragma unroll
    for (int e = 0; e < 50; ++e) o2[e] = make_float2(at((2 * e) / 10, (2 * e) % 10),
                                                    at((2 * e + 1) / 10, (2 * e + 1) % 10));
  } else {
#pragma unroll
    for (int e = 0; e < 100; ++e) out[e] = at(e / 10, e % 10);
  }
  return true;
}

}  // namespace vfisv
