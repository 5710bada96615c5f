// Per-pixel preparation helpers of the paper's pipeline: the empirical
// Stokes-I weight for full-disk maps (Sec. 4.3, Eq. 14) with the continuum
// centre-to-limb variation (Eq. 15), and initial models from the
// filtergrams (Sec. 5): weak-field B and gamma, the azimuth from the line
// wings, the polarisation level, the centre-of-gravity velocity.
#include "common.cuh"

namespace vfisv {

__device__ __forceinline__ float icont_mu(float mu) {
  // Eq. 15, Horner form
  return fmaf(fmaf(fmaf(fmaf(fmaf(0.59943f, mu, -1.89979f), mu, 2.45050f), mu, -1.79238f), mu,
                   1.30590f), mu, 0.33644f);
}

__global__ void limb_weights_kernel(const float* __restrict__ obs, const float* __restrict__ mu,
                                    int64_t npix, int nf, float inv_ic0, float4 inv_sig2,
                                    float* __restrict__ w) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const float* o = obs + p * 4 * nf;
  float ic = -INFINITY;
  float imin = INFINITY;
  for (int k = 0; k < nf; ++k) {
    ic = fmaxf(ic, o[k]);
    imin = fminf(imin, o[k]);
  }
  // wing weights times the squared relative line depth (the outer samples
  // of a spectrum lie in the continuum and carry only noise)
  const float inv_dmax = (ic > imin) ? 1.0f / (ic - imin) : 0.0f;
  // Eq. 14: w_I = 0.7778 |I_cont(mu) - I_cont(x,y)| + 0.3; w_Q = w_U = w_V = 1
  const float wI = fmaf(0.7778f, fabsf(icont_mu(mu[p]) - ic * inv_ic0), 0.3f);
  float* out = w + p * 4 * nf;
  for (int k = 0; k < nf; ++k) {
    out[k] = wI * wI * inv_sig2.x;
    out[nf + k] = inv_sig2.y;
    out[2 * nf + k] = inv_sig2.z;
    out[3 * nf + k] = inv_sig2.w;
  }
}

cudaError_t launch_limb_weights(const float* obs, const float* mu, int64_t npix, int nf,
                                float ic0, const float* sigma4, float* w, cudaStream_t s) {
  const float4 is2 = make_float4(1.0f / (sigma4[0] * sigma4[0]), 1.0f / (sigma4[1] * sigma4[1]),
                                 1.0f / (sigma4[2] * sigma4[2]), 1.0f / (sigma4[3] * sigma4[3]));
  limb_weights_kernel<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(obs, mu, npix, nf,
                                                                      1.0f / ic0, is2, w);
  return cudaGetLastError();
}

// Filter geometry shared by every pixel of a launch: centres (transmission-
// weighted mean wavelength) in increasing order, the original index of each,
// and the wing weights (c_k - cbar)^4 of the azimuth estimate.
constexpr int kGeomMax = 128;  // samples per Stokes parameter the initial models take
struct FilterGeom {
  float c[kGeomMax];
  float wing[kGeomMax];
  int order[kGeomMax];
};

__global__ void filter_geom_kernel(const float* __restrict__ filters, int nf,
                                   const float* __restrict__ wl, int nlam,
                                   FilterGeom* __restrict__ g) {
  __shared__ double cs[kGeomMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < nf; k += blockDim.x >> 5) {
    double sw = 0.0, swx = 0.0;
    for (int i = lane; i < nlam; i += 32) {
      const double t = filters[(size_t)k * nlam + i];
      sw += t;
      swx += t * wl[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
      sw += __shfl_xor_sync(0xffffffffu, sw, o);
      swx += __shfl_xor_sync(0xffffffffu, swx, o);
    }
    if (lane == 0) cs[k] = swx / sw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ord[kGeomMax];
    for (int k = 0; k < nf; ++k) ord[k] = k;
    for (int k = 1; k < nf; ++k)  // insertion sort, stable
      for (int j = k; j > 0 && cs[ord[j]] < cs[ord[j - 1]]; --j) {
        const int t = ord[j];
        ord[j] = ord[j - 1];
        ord[j - 1] = t;
      }
    double mean = 0.0;
    for (int k = 0; k < nf; ++k) mean += cs[k];
    mean /= nf;
    for (int k = 0; k < nf; ++k) {
      g->order[k] = ord[k];
      g->c[k] = (float)cs[ord[k]];
      const double d = cs[ord[k]] - mean;
      g->wing[k] = (float)(d * d * d * d);
    }
  }
}

// Initial models from the filtergrams, one pixel per thread.  mode 0 writes a
// stand-alone model (weak-field B, gamma, psi; centre-of-gravity v; the
// standard guess for the rest); mode 1 edits a model already in `init` the
// paper's way: B and gamma replaced where the polarisation level is below
// pol_thr, psi replaced everywhere.
template <int NF>
__global__ void weak_field_kernel(const float* __restrict__ obs, int64_t npix,
                                  const int64_t* __restrict__ npix_dev,
                                  const FilterGeom* __restrict__ geom, LineK lk, int mode,
                                  float pol_thr, float* __restrict__ init,
                                  float* __restrict__ pol_out) {
  __shared__ FilterGeom G;
  if (threadIdx.x == 0) G = *geom;
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (npix_dev ? *npix_dev : npix)) return;
  const float* o = obs + p * 4 * NF;
  float I[NF], Q[NF], U[NF], V[NF];
  bool finite = true;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    const int j = G.order[k];
    I[k] = o[j];
    Q[k] = o[NF + j];
    U[k] = o[2 * NF + j];
    V[k] = o[3 * NF + j];
    finite = finite && isfinite(I[k]) && isfinite(Q[k]) && isfinite(U[k]) && isfinite(V[k]);
  }
  if (!finite) {  // left to the inversion, which flags it
    if (pol_out) pol_out[p] = NAN;
    if (mode == 0)
      for (int j = 0; j < 10; ++j) init[p * 10 + j] = NAN;
    return;
  }
  // dI/dlambda across the centres: central inside, one-sided at the ends;
  // d2I/dlambda2 at the interior centres from the adjacent slopes
  float d1[NF], d2[NF];
  d1[0] = (I[1] - I[0]) / (G.c[1] - G.c[0]);
  d1[NF - 1] = (I[NF - 1] - I[NF - 2]) / (G.c[NF - 1] - G.c[NF - 2]);
  d2[0] = d2[NF - 1] = 0.0f;
#pragma unroll
  for (int k = 1; k < NF - 1; ++k) {
    d1[k] = (I[k + 1] - I[k - 1]) / (G.c[k + 1] - G.c[k - 1]);
    const float right = (I[k + 1] - I[k]) / (G.c[k + 1] - G.c[k]);
    const float left = (I[k] - I[k - 1]) / (G.c[k] - G.c[k - 1]);
    d2[k] = 2.0f * (right - left) / (G.c[k + 1] - G.c[k - 1]);
  }
  float s11 = 0.0f, sv1 = 0.0f, s22 = 0.0f, sq2 = 0.0f, su2 = 0.0f, wq = 0.0f, wu = 0.0f;
  float ic = I[0], pmax = 0.0f, depth = 0.0f, depthc = 0.0f;
#pragma unroll
  for (int k = 0; k < NF; ++k) {
    s11 = fmaf(d1[k], d1[k], s11);
    sv1 = fmaf(V[k], d1[k], sv1);
    if (k > 0 && k < NF - 1) {
      s22 = fmaf(d2[k], d2[k], s22);
      sq2 = fmaf(Q[k], d2[k], sq2);
      su2 = fmaf(U[k], d2[k], su2);
    }
    wq = fmaf(G.wing[k], Q[k], wq);
    wu = fmaf(G.wing[k], U[k], wu);
    ic = fmaxf(ic, I[k]);
    pmax = fmaxf(pmax, sqrtf(fmaf(Q[k], Q[k], fmaf(U[k], U[k], V[k] * V[k]))));
  }
  // longitudinal field: V = -C B_par dI/dlambda (least squares)
  const float C = lk.cB;
  const float bpar = (s11 > 0.0f) ? -sv1 / (s11 * C) : 0.0f;
  // transverse field: |(Q, U)| = C^2 B_perp^2 / 4 |d2I/dlambda2|
  const float qa = (s22 > 0.0f) ? sq2 / s22 : 0.0f, ub = (s22 > 0.0f) ? su2 / s22 : 0.0f;
  const float bperp = 2.0f * sqrtf(sqrtf(fmaf(qa, qa, ub * ub))) / C;
  // azimuth from the line wings
  float psi = 0.5f * atan2f(wu, wq) * (1.0f / kDeg);
  if (psi < 0.0f) psi += 180.0f;
  const float B = sqrtf(fmaf(bpar, bpar, bperp * bperp));
  const float gamma = atan2f(bperp, bpar) * (1.0f / kDeg);
  const float pol = pmax / ic;
  if (pol_out) pol_out[p] = pol;
  float m[10];
  if (mode == 0) {
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const float d = ic - I[k];
      depth += d;
      depthc = fmaf(d, G.c[k], depthc);
    }
    const float lam = (depth > 0.0f) ? depthc / depth : 0.0f;
    m[0] = B; m[1] = gamma; m[2] = psi;
    m[3] = 10.0f; m[4] = 35.0f; m[5] = 0.25f;
    m[6] = lam / lk.cv;
    m[7] = 0.25f * ic;
    m[8] = 0.75f * ic / lk.mu;
    m[9] = 1.0f;
  } else {
#pragma unroll
    for (int j = 0; j < 10; ++j) m[j] = init[p * 10 + j];
    if (pol < pol_thr) {
      m[0] = B;
      m[1] = gamma;
    }
    m[2] = psi;
  }
  apply_bounds(m);
#pragma unroll
  for (int j = 0; j < 10; ++j) init[p * 10 + j] = m[j];
}

// Batched maps: the start stamp of a call and each map's latency from it.
__global__ void stamp_kernel(unsigned long long* t) { *t = global_ns(); }

__global__ void map_latency_kernel(const unsigned long long* __restrict__ t_done,
                                   const unsigned long long* __restrict__ t0, int nmaps,
                                   float* __restrict__ ms) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmaps) return;
  const unsigned long long t = t_done[m];
  ms[m] = (t >= *t0) ? (float)((double)(t - *t0) * 1e-6) : 0.0f;  // empty maps: 0
}

cudaError_t launch_stamp(unsigned long long* t, cudaStream_t s) {
  stamp_kernel<<<1, 1, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_map_latency(const unsigned long long* t_done, const unsigned long long* t0,
                               int nmaps, float* ms, cudaStream_t s) {
  map_latency_kernel<<<(nmaps + 127) / 128, 128, 0, s>>>(t_done, t0, nmaps, ms);
  return cudaGetLastError();
}

// The same estimates for many samples per Stokes parameter (spectrograph-
// shaped inputs), with the sample count at run time: one pixel per thread,
// two passes over the observables (I_c first, then the sums), the three-point
// window of the differences carried along.
__global__ void weak_field_many_kernel(const float* __restrict__ obs, int64_t npix,
                                       const int64_t* __restrict__ npix_dev, int nf,
                                       const FilterGeom* __restrict__ geom, LineK lk, int mode,
                                       float pol_thr, float* __restrict__ init,
                                       float* __restrict__ pol_out) {
  __shared__ FilterGeom G;
  for (int k = threadIdx.x; k < nf; k += blockDim.x) {
    G.c[k] = geom->c[k];
    G.wing[k] = geom->wing[k];
    G.order[k] = geom->order[k];
  }
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (npix_dev ? *npix_dev : npix)) return;
  const float* o = obs + p * 4 * nf;
  float ic = -INFINITY;
  bool finite = true;
  for (int j = 0; j < 4 * nf; ++j) finite = finite && isfinite(o[j]);
  if (!finite) {
    if (pol_out) pol_out[p] = NAN;
    if (mode == 0)
      for (int j = 0; j < 10; ++j) init[p * 10 + j] = NAN;
    return;
  }
  float imin = INFINITY;
  for (int k = 0; k < nf; ++k) {
    ic = fmaxf(ic, o[k]);
    imin = fminf(imin, o[k]);
  }
  // wing weights times the squared relative line depth (the outer samples
  // of a spectrum lie in the continuum and carry only noise)
  const float inv_dmax = (ic > imin) ? 1.0f / (ic - imin) : 0.0f;
  float s11 = 0.0f, sv1 = 0.0f, s22 = 0.0f, sq2 = 0.0f, su2 = 0.0f, wq = 0.0f, wu = 0.0f;
  float pmax = 0.0f, depth = 0.0f, depthc = 0.0f;
  // window: previous, current, next (in increasing centre order)
  float Ip = 0.0f, Ic0 = o[G.order[0]], In = o[G.order[1]];
  for (int k = 0; k < nf; ++k) {
    const int j = G.order[k];
    const float Q = o[nf + j], U = o[2 * nf + j], V = o[3 * nf + j];
    float d1;
    if (k == 0) {
      d1 = (In - Ic0) / (G.c[1] - G.c[0]);
    } else if (k == nf - 1) {
      d1 = (Ic0 - Ip) / (G.c[k] - G.c[k - 1]);
    } else {
      d1 = (In - Ip) / (G.c[k + 1] - G.c[k - 1]);
      const float right = (In - Ic0) / (G.c[k + 1] - G.c[k]);
      const float left = (Ic0 - Ip) / (G.c[k] - G.c[k - 1]);
      const float d2 = 2.0f * (right - left) / (G.c[k + 1] - G.c[k - 1]);
      s22 = fmaf(d2, d2, s22);
      sq2 = fmaf(Q, d2, sq2);
      su2 = fmaf(U, d2, su2);
    }
    s11 = fmaf(d1, d1, s11);
    sv1 = fmaf(V, d1, sv1);
    const float rd = (ic - Ic0) * inv_dmax;
    const float wk = G.wing[k] * rd * rd;
    wq = fmaf(wk, Q, wq);
    wu = fmaf(wk, U, wu);
    pmax = fmaxf(pmax, sqrtf(fmaf(Q, Q, fmaf(U, U, V * V))));
    const float d = ic - Ic0;
    depth += d;
    depthc = fmaf(d, G.c[k], depthc);
    Ip = Ic0;
    Ic0 = In;
    In = (k + 2 < nf) ? o[G.order[k + 2]] : 0.0f;
  }
  const float C = lk.cB;
  const float bpar = (s11 > 0.0f) ? -sv1 / (s11 * C) : 0.0f;
  const float qa = (s22 > 0.0f) ? sq2 / s22 : 0.0f, ub = (s22 > 0.0f) ? su2 / s22 : 0.0f;
  const float bperp = 2.0f * sqrtf(sqrtf(fmaf(qa, qa, ub * ub))) / C;
  float psi = 0.5f * atan2f(wu, wq) * (1.0f / kDeg);
  if (psi < 0.0f) psi += 180.0f;
  const float B = sqrtf(fmaf(bpar, bpar, bperp * bperp));
  const float gamma = atan2f(bperp, bpar) * (1.0f / kDeg);
  const float pol = pmax / ic;
  if (pol_out) pol_out[p] = pol;
  float m[10];
  if (mode == 0) {
    const float lam = (depth > 0.0f) ? depthc / depth : 0.0f;
    m[0] = B; m[1] = gamma; m[2] = psi;
    m[3] = 10.0f; m[4] = 35.0f; m[5] = 0.25f;
    m[6] = lam / lk.cv;
    m[7] = 0.25f * ic;
    m[8] = 0.75f * ic / lk.mu;
    m[9] = 1.0f;
  } else {
    for (int j = 0; j < 10; ++j) m[j] = init[p * 10 + j];
    if (pol < pol_thr) {
      m[0] = B;
      m[1] = gamma;
    }
    m[2] = psi;
  }
  apply_bounds(m);
  for (int j = 0; j < 10; ++j) init[p * 10 + j] = m[j];
}

size_t filter_geom_bytes() { return sizeof(FilterGeom); }

cudaError_t launch_weak_field(const float* obs, int64_t npix, const int64_t* npix_dev,
                              const float* filters, int nf, const float* wl, int nlam,
                              const LineK& lk, int mode, float pol_thr, void* geom, float* init,
                              float* pol_out, cudaStream_t s) {
  if (nf < 3 || nf > kGeomMax) return cudaErrorInvalidValue;
  filter_geom_kernel<<<1, 256, 0, s>>>(filters, nf, wl, nlam, (FilterGeom*)geom);
  const unsigned grid = (unsigned)((npix + 255) / 256);
  const FilterGeom* g = (const FilterGeom*)geom;
  if (nf > 8) {
    weak_field_many_kernel<<<grid, 256, 0, s>>>(obs, npix, npix_dev, nf, g, lk, mode, pol_thr,
                                                init, pol_out);
    return cudaGetLastError();
  }
  switch (nf) {
    case 3: weak_field_kernel<3><<<grid, 256, 0, s>>>(obs, npix, npix_dev, g, lk, mode, pol_thr, init, pol_out); break;
    case 4: weak_field_kernel<4><<<grid, 256, 0, s>>>(obs, npix, npix_dev, g, lk, mode, pol_thr, init, pol_out); break;
    case 5: weak_field_kernel<5><<<grid, 256, 0, s>>>(obs, npix, npix_dev, g, lk, mode, pol_thr, init, pol_out); break;
    case 6: weak_field_kernel<6><<<grid, 256, 0, s>>>(obs, npix, npix_dev, g, lk, mode, pol_thr, init, pol_out); break;
    case 7: weak_field_kernel<7><<<grid, 256, 0, s>>>(obs, npix, npix_dev, g, lk, mode, pol_thr, init, pol_out); break;
    default: weak_field_kernel<8><<<grid, 256, 0, s>>>(obs, npix, npix_dev, g, lk, mode, pol_thr, init, pol_out); break;
  }
  return cudaGetLastError();
}

}  // namespace vfisv
