/*
 * vfisv.h -- C ABI of the GB300 Milne-Eddington Stokes inversion library
 * (libvfisv.so).
 *
 * The library computes, for many independent pixels, the per-pixel hot path
 * of the VFISV inversion (Borrero et al., "VFISV: Very Fast Inversion of the
 * Stokes Vector for the Helioseismic and Magnetic Imager"):
 *   - Milne-Eddington (Unno-Rachkovsky) synthesis of (I, Q, U, V) of a
 *     normal Zeeman triplet (Sec. 3.1, Eq. 7) from the Voigt and
 *     Faraday-Voigt functions (Sec. 3.2, Eqs. 8-9), convolved with the
 *     instrument's filter transmission profiles;
 *   - its analytic Jacobian (Sec. 4.4);
 *   - Levenberg-Marquardt minimisation of chi-square (Sec. 2, Eqs. 1-6;
 *     Sec. 4.2, Table 2; Sec. 4.4, Fig. 6);
 *   - the learned initial guess (Sec. 5) as a 24-256-256-256-11 network.
 *
 * Conventions shared by every entry point
 *   - Pointers may be device memory or host memory (pageable or pinned);
 *     the library detects which.  Host buffers are staged through device
 *     workspaces owned by the handle and the call returns after the results
 *     are back in host memory.  With device buffers the call is
 *     asynchronous on `stream`.
 *   - All arrays are C-contiguous, caller-owned; the library never frees or
 *     retains caller memory beyond the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).
 *   - Return value: VFISV_OK (0) or a negative VFISV_E_* code.  Problems
 *     of single pixels never fail a call; they are reported per pixel in
 *     `status_out`.
 *
 * Parameter vector of one pixel, float32[10], in this order (Sec. 2 with
 * the macroturbulence dropped):
 *   0 B [G]   1 gamma [deg]   2 psi [deg]   3 eta0   4 dlambdaD [mA]
 *   5 a       6 v_los [km/s, positive = redshift]    7 S0   8 S1
 *   9 alpha (magnetic filling factor)
 * Observables of one pixel, float32[4][nfilt]: Stokes I, Q, U, V at each
 * filter position, in that order.
 */
#ifndef VFISV_H
#define VFISV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VFISV_NPARAM 10

/* Initial-guess network: 24 inputs (the observables divided by the largest
 * Stokes I sample, standardised), three GELU hidden layers of 256, 11
 * outputs (B, cos gamma, sin 2psi, cos 2psi, ln eta0, dlambdaD, a, v_los,
 * S0/Ic, S1/Ic standardised, and a confidence = predicted log mean squared
 * error of the other ten).  Its float32 parameter blob holds, in order:
 *   W0[24][256] b0[256] W1[256][256] b1[256] W2[256][256] b2[256]
 *   W3[256][11] b3[11]  (weights [fan_in][fan_out]: y = x W + b)
 *   in_mean[24] in_std[24] out_mean[10] out_std[10]  (standardisation)
 * The first VFISV_NN_NTRAIN floats are trained; the rest are statistics of
 * the training set. */
#define VFISV_NN_NIN 24
#define VFISV_NN_NHID 256
#define VFISV_NN_NOUT 11
#define VFISV_NN_NTRAIN 140811
#define VFISV_NN_NBLOB 140879

enum {
  VFISV_OK = 0,
  VFISV_E_ARG = -1,         /* null pointer or invalid argument value */
  VFISV_E_SIZE = -2,        /* a size is out of the supported range */
  VFISV_E_UNSUPPORTED = -3, /* nfilt not compiled into this kernel */
  VFISV_E_CUDA = -4,        /* a CUDA runtime call failed */
  VFISV_E_DEVICE = -5,      /* a kernel reported an internal error */
  VFISV_E_NOMEM = -6,       /* a workspace allocation failed */
  VFISV_E_CAPTURE = -7      /* a workspace would have to grow during capture */
};

/* Per-pixel status codes written to status_out. */
enum {
  VFISV_PIX_CONVERGED = 0, /* chi2 stopped decreasing (see vfisv_config) */
  VFISV_PIX_MAXITER = 1,   /* iteration cap reached first */
  VFISV_PIX_STALLED = 2,   /* damping exceeded 1e12: no decrease possible */
  VFISV_PIX_BAD_INPUT = 3, /* non-finite observable, weight or initial model,
                              or all weights zero; outputs hold the guess */
  VFISV_PIX_NAN_STATE = 4  /* synthesis at the initial model not finite */
};

/* A normal Zeeman triplet (Sec. 3.1).  The sigma components sit at
 * +-dlambda_B = +-4.66685e-10 * geff * lambda0_A^2 * B  [mA]  (Eq. 7), the
 * Doppler shift is lambda0 * v / c.  mu is the heliocentric angle cosine
 * multiplying S1 in the Milne-Eddington solution. */
typedef struct {
  double lambda0_A;
  double geff;
  double mu;
} vfisv_line;

/* Levenberg-Marquardt controls (Sec. 4.2).
 *   max_iter   cap on trial steps (solves) per pixel; the paper runs a fixed
 *              count (30) -- here a pixel also stops when converged.
 *   free_mask  bit p set = parameter p is free.  Bit 9 frees the filling
 *              factor alpha (Sec. 2; default held at 1): the model mixes the
 *              magnetic and the non-magnetic (B = 0) profile, alpha in
 *              [0, 1], 10 parameters in the solve and the covariance; taken
 *              by the 6-filter path with the FP64 solve and no restarts
 *              (else VFISV_E_UNSUPPORTED), not by vfisv_invert_noalloc.
 *   conv_rtol  converged when a successful step lowers chi2 by less than
 *              conv_rtol relative while the damping used was <= conv_eps.
 *   eps0       initial damping.
 *   restarts   randomised restarts (Sec. 4.2), a bit mask; 0 = off (a pixel
 *              stops when converged).  With any bit set every pixel runs
 *              exactly max_iter iterations and a restart is due
 *                bit 0  when a step meets the convergence test or the pixel
 *                       stalls (else such a pixel stops there),
 *                bit 1  (the paper's (a)) at iteration 10 if the best chi2 is
 *                       not below a tenth of the initial chi2,
 *                bit 2  (the paper's (b)) after 5 failed trials in a row;
 *              7 = the paper's rule.  A restart replaces the next trial: the
 *              best model of all segments, perturbed as vfisv_restart_models
 *              does with k = the pixel's restart count, starts a new segment
 *              whatever its chi2, with the damping reset to eps0; it counts
 *              as one iteration.  Outputs are the best model of all segments,
 *              its chi2 and covariance; status CONVERGED if any segment
 *              converged, else STALLED if any stalled, else MAXITER.
 *              The pixel number of the perturbations is the pixel's index in
 *              the call.  max_iter must stay below 2^20 with restarts.
 *   seed       key of the perturbations.
 *   wfa_pol    initialisation from the filtergrams (Sec. 5), 0 = off.
 *              Where an inversion starts without given models (vfisv_invert
 *              with init == NULL, the re-inversion stage of vfisv_invert_nn),
 *              > 0 starts from the models of vfisv_init_models instead of the
 *              standard guess (both the 6-filter and the spectrograph-shaped
 *              path).  In the first stage of vfisv_invert_nn, > 0
 *              combines the network's guess the paper's way: B and gamma from
 *              the weak-field estimate where the polarisation level is below
 *              wfa_pol (the paper: 0.06), the wing azimuth everywhere, the
 *              network's values for the rest.
 *   fast_solve 0 (default): the damped solve, the covariance and the chi2
 *              acceptance sum in FP64.  1: the solve and the covariance in
 *              double-float arithmetic (pairs of FP32 numbers, ~48 bits) and
 *              chi2 by a compensated FP32 sum -- no FP64 on the fast path,
 *              whose FP64 pipe issues 2 FMAs per SM per clock on GB300
 *              against 128 in FP32.  Not the paper's precision: opt-in.
 *   hess_reuse Hessian reuse near the minimum (Sec. 4.4), 0 = off: when an
 *              accepted step lowered chi2 by less than hess_reuse relative,
 *              and so did the previous accepted step, J^T W J is kept from
 *              the previous model and only J^T W r is rebuilt; the
 *              covariance comes from the matrix in use.
 * vfisv_config_default() fills: 50, 0x1FF, 1e-4, 1.0, 1.0, 0, 0, 0.0, 0.0, 0. */
typedef struct {
  int32_t max_iter;
  uint32_t free_mask;
  double conv_rtol;
  double conv_eps;
  double eps0;
  int32_t restarts;
  uint64_t seed;
  double hess_reuse;
  double wfa_pol;
  int32_t fast_solve;
} vfisv_config;

typedef struct vfisv_handle vfisv_handle;

/* Create a handle bound to CUDA device `device` (it becomes current on the
 * calling thread for every call made with the handle).  Owns workspaces,
 * the work-queue counter and the Weideman coefficients. */
int vfisv_create(vfisv_handle** out, int device);
void vfisv_destroy(vfisv_handle* h);
void vfisv_config_default(vfisv_config* cfg);
const char* vfisv_strerror(int code);

/* Voigt and Faraday-Voigt functions H(a,u) + i F(a,u) = w(u + i a) of n
 * points (Sec. 3.2), a >= 0:
 *   method 0  the Weideman rational series the synthesis kernels use;
 *   method 1  the paper's Taylor table, first order (Eqs. 8-9, 12-13):
 *             H, F tabulated at u = 0..20 step 0.04 and a = 0..5 step 0.05,
 *             extrapolated from the nearest node;
 *   method 2  the same to second order (Eqs. 10-13).
 * Points outside the table use the rational series.  Arrays float32[n]. */
int vfisv_voigt(vfisv_handle* h, const float* a, const float* u, int64_t n, int32_t method,
                float* H, float* F, void* stream);

/* Many maps in one persistent launch (the uneven serving mix): the pixels of
 * nmaps maps concatenated in obs [npix][4][nfilt], map m holding pixels
 * map_off[m] .. map_off[m+1]-1 (map_off: host int64 [nmaps+1], map_off[0] =
 * 0, non-decreasing, npix = map_off[nmaps]); weights [nmaps][4][nfilt] are
 * per map (w^2/sigma^2 shared by the map's pixels).  Any nfilt vfisv_invert
 * takes (6 filter positions, or the wide instrument path).  Outputs as
 * vfisv_invert, plus latency_ms [nmaps] (optional): for each map, the time
 * from the start of this call's first kernel to the retirement of the map's
 * last pixel by the LM kernel, read from the GPU's global timer (the
 * covariance pass that follows is not included; an empty map reads 0).
 * The offsets are copied into a pinned buffer of the handle, which a
 * captured graph keeps reading on every replay: a later batch call on the
 * same handle changes what the replays see.  Host or device buffers. */
int vfisv_invert_batch(vfisv_handle* h, const float* obs, const float* weights,
                       const int64_t* map_off, int32_t nmaps, const float* filters,
                       int32_t nfilt, const float* wl_mA, int32_t nlam, const vfisv_line* line,
                       const float* init, const vfisv_config* cfg, float* params_out,
                       float* chi2_out, int32_t* iters_out, int32_t* status_out, float* cov_out,
                       float* latency_ms, void* stream);

/* Initial models from the filtergrams (Sec. 5; the paper's methods are
 * cited, not printed -- this is one reading of them).  For each pixel of
 * obs [npix][4][nfilt] (3 <= nfilt <= 128; filters [nfilt][nlam] on wl_mA, any
 * order of centres):
 *   c_k      filter centres sum T_k x / sum T_k, taken in increasing order;
 *   B_par    least-squares fit of V_k = -C B_par dI/dlambda_k, the derivative
 *            by differences across the centres (central inside, one-sided
 *            at the ends), C = 4.66685e-10 g lambda0^2 mA/G (Eq. 7);
 *   B_perp   least-squares fit of |(Q_k, U_k)| = C^2 B_perp^2 / 4 |d2I/dlambda2_k|
 *            over the interior centres;
 *   psi      azimuth from the line wings: 2 psi = atan2(sum w_k U_k,
 *            sum w_k Q_k), w_k = (c_k - mean c)^4, times the squared relative
 *            line depth ((I_c - I_k) / max_j (I_c - I_j))^2 when nfilt > 8
 *            (spectra that reach into the continuum);
 *   B = hypot(B_par, B_perp), gamma = atan2(B_perp, B_par);
 *   v        centre of gravity of the line depth I_c - I_k over the centres;
 *   eta0 = 10, dlambdaD = 35 mA, a = 0.25, S0 = 0.25 I_c, S1 = 0.75 I_c / mu,
 *   alpha = 1 (I_c = largest Stokes I sample); the model bounds applied.
 * init_out [npix][10]; pol_out (optional) [npix] = max_k |(Q,U,V)_k| / I_c,
 * the polarisation level the paper's 6 % switch uses.  A pixel with a
 * non-finite observable gets a NaN model and pol (the inversion then flags
 * it BAD_INPUT).  Host or device buffers. */
int vfisv_init_models(vfisv_handle* h, const float* obs, int64_t npix, const float* filters,
                      int32_t nfilt, const float* wl_mA, int32_t nlam, const vfisv_line* line,
                      float* init_out, float* pol_out, void* stream);

/* The perturbation of a randomised restart (Sec. 4.2), in bulk: models_out
 * [n][10] = restart number k (1 <= k < 2^20) of pixels pixel0 .. pixel0+n-1
 * from models [n][10].  With r = 2u - 1 and u uniform in [0, 1), the free
 * parameters among B, gamma, psi, eta0, dlambdaD, a, v move by r*k times
 * 150 G, 10 deg, 15 deg, (ln eta0) 0.25, 4 mA, 0.05, 0.25 km/s; S0, S1,
 * alpha and held parameters (free_mask bit clear) are copied; the model
 * bounds of vfisv_invert are applied.  u is the top 53 bits of SplitMix64
 * (Steele, Lea & Flood 2014) output number (pixel << 24 | k << 4 | p) of the
 * stream keyed by `seed`, p the parameter's index.  Host or device buffers.
 * pixel0 + n <= 2^40. */
int vfisv_restart_models(vfisv_handle* h, const float* models, int64_t n, int64_t pixel0,
                         int32_t k, uint32_t free_mask, uint64_t seed, float* models_out,
                         void* stream);

/* Weights for full-disk maps (Sec. 4.3): w_I = 0.7778 |I_cont(mu) - I_c| + 0.3
 * (Eq. 14) with I_cont(mu) the quintic centre-to-limb law of Eq. 15 and I_c
 * the pixel's largest Stokes I sample divided by the disk-centre continuum
 * ic0; w_Q = w_U = w_V = 1.  Writes weights_out[npix][4][nfilt] = w^2 /
 * sigma^2 with sigma4 (host float[4]) the noise of I, Q, U, V; mu[npix] is the
 * heliocentric angle cosine of each pixel. */
int vfisv_limb_weights(vfisv_handle* h, const float* obs, const float* mu, int64_t npix,
                       int32_t nfilt, float ic0, const float* sigma4, float* weights_out,
                       void* stream);

/* Whole-map CUDA graphs.  vfisv_graph_begin starts a (relaxed-mode) capture
 * on `stream` (not the legacy NULL stream); every vfisv_* call made with the
 * handle and device buffers until vfisv_graph_end is recorded instead of
 * run, and vfisv_graph_end instantiates the graph.  Workspaces cannot grow
 * while capturing (VFISV_E_CAPTURE): make one uncaptured call with the same
 * sizes first.  vfisv_graph_launch replays it (same buffers, new contents);
 * calls that synchronise (vfisv_check, host buffers, vfisv_autotune) are not
 * capturable. */
typedef struct vfisv_graph vfisv_graph;
int vfisv_graph_begin(vfisv_handle* h, void* stream);
int vfisv_graph_end(vfisv_handle* h, void* stream, vfisv_graph** out);
int vfisv_graph_launch(vfisv_graph* g, void* stream);
/* Number of kernel launches one replay of the graph performs (kernel nodes,
 * child graphs included), written to *count.  VFISV_E_ARG for a null graph
 * or count. */
int vfisv_graph_kernels(const vfisv_graph* g, int64_t* count);
void vfisv_graph_destroy(vfisv_graph* g);

/* Autotuner for the launch shape of the filter-position LM kernel (the
 * workload asks for pixels per CTA and threads per pixel to be tuned): time
 * an inversion of the given sample (arguments as vfisv_invert, no
 * covariance) with 64, 128 and 256 threads per CTA and 1, 2 and 4 threads
 * per pixel, and with the warp-specialised kernel (384 threads per CTA, one
 * pixel per thread of its two consumer warpgroups, one CTA per SM), keep the
 * fastest shape for this handle's later inversions and return it in
 * best_block (threads per CTA) and best_tpp (threads per pixel, may be
 * NULL); ms_out (may be NULL) receives the ten times: ms_out[3 * i + j] for
 * tpp = {1, 2, 4}[i], block = {64, 128, 256}[j], then ms_out[9] for 384 x 1.
 * With tpp threads per pixel the lanes of a pixel split its wavelength
 * points: a pass has tpp times as many threads, so small maps (fewer pixels
 * than resident slots) finish sooner, while the solve and the normal
 * equations are repeated on every lane of the pixel.  The warp-specialised
 * kernel runs the wavelength pass in one warpgroup and the chi2, normal
 * equations and FP64 solve in the other two, handing the filtered rows over
 * through tensor memory; it takes the default configuration (restarts, a
 * free filling factor and fast_solve run the 128 x 1 kernel instead).
 * Results do not
 * depend on the shape beyond FP32 summation order.  Synchronises `stream`. */
int vfisv_autotune(vfisv_handle* h, const float* obs, const float* weights,
                   int32_t weights_per_pixel, const float* filters, int32_t nfilt,
                   const float* wl_mA, int32_t nlam, const vfisv_line* line,
                   const vfisv_config* cfg, int64_t npix, int32_t* best_block, int32_t* best_tpp,
                   float* ms_out /*[10]*/, void* stream);

/* Set the launch shape of the handle's filter-position LM kernel directly:
 * block in {64, 128, 256} threads per CTA with tpp in {1, 2, 4} threads per
 * pixel, or block = 384 with tpp = 1 for the warp-specialised kernel
 * (default 128 x 1).  VFISV_E_ARG for any other value. */
int vfisv_set_launch_shape(vfisv_handle* h, int32_t block, int32_t tpp);

/* Persistent launches of this handle (the LM, wide, covariance and network
 * kernels) use at most `nsm` SMs; 0 (the default) lets them take every SM.
 * For two handles inverting side by side on concurrent streams: a
 * persistent LM launch fills every SM's register file, so without a split
 * the first launch takes the GPU and the other waits for it.  A graph captures the grids in force
 * at capture time.  VFISV_E_ARG for nsm < 0. */
int vfisv_set_sm_limit(vfisv_handle* h, int32_t nsm);

/* Host-buffer pipeline depth.  vfisv_invert and vfisv_invert_nn given host
 * observations for 2^20 pixels or more (no restarts, not capturing) copy the
 * per-pixel rows in and out in `chunks` chunks on two copy streams of the
 * handle, double-buffered on the device, while the caller's stream inverts
 * the previous chunk; the outputs are those of one call over the whole map.
 * With 3 or more chunks the first and last hold an eighth of the rows of
 * each middle chunk (only their copies are not hidden).  chunks = 0 stages
 * the whole map before the inversion instead; default 3.
 * VFISV_E_ARG for chunks < 0 or > 64. */
int vfisv_set_pipeline_chunks(vfisv_handle* h, int32_t chunks);

/* Synchronise `stream` and report any error a kernel of this handle flagged
 * on the device since the last check (VFISV_E_DEVICE) or a CUDA error.  A
 * device error is a bounded wait (about a second) that gave up: the filter
 * table's copy into shared memory, a network operand copy or tensor-core
 * completion, a filtered-row buffer of the one-warpgroup LM kernel, or a
 * producer/consumer hand-off of the warp-specialised LM kernel.  The kernel
 * then stops and returns, so the context stays usable, but the outputs of
 * the calls since the last check are not valid.  The error words are
 * cleared. */
int vfisv_check(vfisv_handle* h, void* stream);

/* Work done by this handle's filter-position LM launches (nfilt = 6; the
 * spectrograph-shaped path is not counted) since the handle was created or
 * last reset, for measuring the method's own work (Sec. 4.4, Fig. 6):
 *   out[0] fused passes: one per trial model plus one per starting model
 *   out[1] accepted trials, each followed by a J^T W J / J^T W r build
 *   out[2] pixels retired
 *   out[3] wavelength points evaluated: passes x grid points in use (the
 *          packed filter table leaves out the grid points of least weight
 *          while every filter keeps all but 2^-24 of its summed |weight|,
 *          which moves a filtered value by at most one FP32 rounding)
 * Synchronises `stream` first; reset != 0 zeroes the counters afterwards.
 * Replays of a captured graph add to them like direct calls. */
int vfisv_counters(vfisv_handle* h, void* stream, uint64_t* out, int32_t reset);  /* out[4] */

/* Milne-Eddington synthesis through the filters (Secs. 3.1-3.2).
 *   params   float32[npix][10]   model (alpha in [0,1] honoured)
 *   filters  float32[nfilt][nlam] transmission T_k(x_i)
 *   wl_mA    float32[nlam]       x_i = lambda_i - lambda0 in mA
 *   line     the triplet
 *   stokes   float32[npix][4][nfilt] output: S_jk = sum_i T_k(x_i) S_j(x_i)
 * 1 <= nfilt <= 8 (filter positions, one pixel per thread), or 9 <= nfilt <=
 * 128 narrow instrument profiles (spectrograph-shaped inputs, one pixel per
 * warp: nlam <= 1024, each profile non-zero over at most 32 consecutive
 * points, else VFISV_E_UNSUPPORTED on the device error word);
 * 1 <= nlam <= 4096, npix >= 0 (0 is a no-op). */
int vfisv_synth(vfisv_handle* h, const float* params, int64_t npix,
                const float* filters, int32_t nfilt, const float* wl_mA,
                int32_t nlam, const vfisv_line* line, float* stokes,
                void* stream);

/* Levenberg-Marquardt inversion of every pixel (Secs. 2 and 4).
 *   obs        float32[npix][4][nfilt] observed Stokes vector
 *   weights    w_ij^2 / sigma_ij^2 of Eq. 1: float32[npix][4][nfilt] if
 *              weights_per_pixel, else float32[4][nfilt] for all pixels;
 *              zero marks missing data (Sec. 4.3)
 *   init       float32[npix][10] initial models, or NULL for the standard
 *              guess B=500 G, gamma=60, psi=45, eta0=10, dlambdaD=35 mA,
 *              a=0.25, v=0, S0=0.25 Ic, S1=0.75 Ic/mu (Ic = largest I sample)
 *   params_out float32[npix][10] best model (alpha = 1)
 *   chi2_out   float32[npix]     Eq. 1 at params_out (dof = 4 nfilt - F)
 *   iters_out  int32[npix]       trial steps taken
 *   status_out int32[npix]       VFISV_PIX_*
 *   cov_out    float32[npix][10][10] (J^T W J)^+ at params_out in parameter
 *              units (zero rows/columns for held parameters), or NULL
 * nfilt == 6 (filter positions, one pixel per thread slot; every option of
 * vfisv_config), or 9 <= nfilt <= 128 narrow instrument profiles
 * (spectrograph-shaped inputs, one pixel per warp, nlam <= 1024, profiles
 * non-zero over at most 32 consecutive points; restarts, hess_reuse,
 * fast_solve and a free filling factor are VFISV_E_UNSUPPORTED there);
 * other nfilt: VFISV_E_UNSUPPORTED.  1 <= nlam <= 4096. */
int vfisv_invert(vfisv_handle* h, const float* obs, const float* weights,
                 int32_t weights_per_pixel, const float* filters,
                 int32_t nfilt, const float* wl_mA, int32_t nlam,
                 const vfisv_line* line, const float* init,
                 const vfisv_config* cfg, int64_t npix, float* params_out,
                 float* chi2_out, int32_t* iters_out, int32_t* status_out,
                 float* cov_out, void* stream);

/* Initialise a network blob for training (Sec. 5): weights uniform in
 * +-sqrt(6/fan_in) from a counter-based hash of (seed, index), biases zero,
 * and the standardisation statistics (mean, standard deviation; FP64
 * accumulation) of the n training pairs.
 *   blob    float32[VFISV_NN_NBLOB] output
 *   obs     float32[n][24] observables of the training profiles
 *   params  float32[n][10] their generating models */
int vfisv_nn_init(vfisv_handle* h, float* blob, const float* obs, const float* params,
                  int64_t n, uint64_t seed, void* stream);

/* Train in place: Adam (beta1 0.9, beta2 0.999, eps 1e-8) with cosine
 * learning-rate decay from lr0 to 0 over epochs * floor(n / batch) steps,
 * minibatches drawn by a per-epoch affine permutation of the training set.
 * Loss = mean squared error of the 10 standardised targets + squared error
 * of the confidence output against log(mean squared error + 1e-4).
 * batch must be a positive multiple of 512; n < 2^31.
 *   loss_hist  float32[epochs * floor(n / batch)] per-step loss, or NULL */
int vfisv_nn_train(vfisv_handle* h, float* blob, const float* obs, const float* params,
                   int64_t n, int32_t batch, int32_t epochs, float lr0, uint64_t seed,
                   float* loss_hist, void* stream);

/* Loss and gradient for one batch of n pairs (the training kernels' forward
 * and backward passes, BF16 operands, FP32 accumulation).
 *   grad_out  float32[VFISV_NN_NTRAIN] dL/d(weights, biases), blob layout
 *   loss_out  float32[1]
 * 1 <= n <= 2^20. */
int vfisv_nn_grad(vfisv_handle* h, const float* blob, const float* obs, const float* params,
                  int64_t n, float* grad_out, float* loss_out, void* stream);

/* Network initial guesses for npix pixels (Sec. 5), in one fused kernel:
 * features, the four layers (BF16 operands rounded to nearest, FP32
 * accumulation, FP32 bias and GELU), decoding.
 *   init_out  float32[npix][10] models decoded from the outputs (alpha = 1)
 *   conf_out  float32[npix] confidence output, or NULL
 *   raw_out   float32[npix][11] raw (standardised) outputs, or NULL */
int vfisv_nn_infer(vfisv_handle* h, const float* blob, const float* obs, int64_t npix,
                   const vfisv_line* line, float* init_out, float* conf_out, float* raw_out,
                   void* stream);

/* Mixed inversion (Sec. 5: the network supplies an initial guess only; LM
 * from the standard guess stays the fallback): network guess and confidence
 * output, then
 *   - pixels with confidence output > conf_route (the network's estimate of
 *     its own log mean squared error in standardised units: an uncertain
 *     guess) skip the LM run from the guess;
 *   - the others run LM from the guess with cfg_nn;
 *   - every routed pixel, and every pixel that ends with chi2 > chi2_flag (or,
 *     with flag_unconverged, that did not converge; STALLED counts as
 *     converged), is inverted from the standard guess with cfg_plain; a
 *     re-inverted pixel keeps the lower-chi2 of its results (a routed pixel
 *     the plain one).
 * conf_route = +INFINITY disables routing (every pixel runs LM from the
 * guess); NaN is VFISV_E_ARG.  Arguments as vfisv_invert; iters_out counts
 * the steps of both runs; flagged_out (int32[npix], or NULL) marks the
 * re-inverted pixels, routed ones included. */
int vfisv_invert_nn(vfisv_handle* h, const float* blob, const float* obs, const float* weights,
                    int32_t weights_per_pixel, const float* filters, int32_t nfilt,
                    const float* wl_mA, int32_t nlam, const vfisv_line* line,
                    const vfisv_config* cfg_nn, const vfisv_config* cfg_plain,
                    double chi2_flag, int32_t flag_unconverged, double conf_route, int64_t npix,
                    float* params_out, float* chi2_out,
                    int32_t* iters_out, int32_t* status_out, float* cov_out,
                    int32_t* flagged_out, void* stream);

/* Allocation-free variant of vfisv_invert.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * that runs inside a host framework owning all device memory through its
 * own pool (a cudaMalloc would bypass the pool's accounting and its hard
 * cap), and real-time pipelines that allocate everything up front because a
 * cudaMalloc or cudaFree can synchronise the device and stall their other
 * streams.  It takes no handle and allocates nothing: the kernel's scratch
 * (pixel-slot normal equations, work-queue counter, error word, packed
 * filter table) is a fixed array of VFISV_NOALLOC_SCRATCH_BYTES (about
 * 8.1 MiB) compiled into the library; every GPU that loads the library
 * holds it until the process exits.
 *   - All pointers must be device memory; arguments and outputs are those
 *     of vfisv_invert, on the current CUDA device, asynchronous on `stream`.
 *   - nlam <= VFISV_NOALLOC_MAX_NLAM (4096) and nfilt == 6, else
 *     VFISV_E_SIZE / VFISV_E_UNSUPPORTED; cfg->restarts and cfg->wfa_pol must be 0.  Any npix works: at most
 *     VFISV_NOALLOC_MAX_SLOTS pixels are resident at once and the others
 *     queue behind them.
 *   - The first call on a device looks up the array's device address and
 *     uploads the kernel's constants (blocking calls): make that first call
 *     before any stream capture.  First calls from several host threads at
 *     once are safe (the set-up runs once per device, under a lock).
 *   - Every call, from any thread or stream, shares the one array: calls
 *     whose kernels overlap on the GPU race and corrupt each other's
 *     results; serialise them (one stream, or events).  Each call clears the
 *     work-queue counter and the device error word itself, on `stream`; the
 *     rest of the array is overwritten before it is read.
 *   - Per-pixel problems go to status_out as in vfisv_invert.  A device-side
 *     failure of the call itself (a bounded wait in the kernel that gave up;
 *     its outputs are then not valid) is recorded in the array's error word:
 *     read it with vfisv_noalloc_check before the next call.
 *   - The call uses every SM of the device (no handle, so no
 *     vfisv_set_sm_limit). */
#define VFISV_NOALLOC_MAX_NLAM 4096
#define VFISV_NOALLOC_MAX_SLOTS 38912
#define VFISV_NOALLOC_SCRATCH_BYTES 8536576
int vfisv_invert_noalloc(const float* obs, const float* weights, int32_t weights_per_pixel,
                         const float* filters, int32_t nfilt, const float* wl_mA, int32_t nlam,
                         const vfisv_line* line, const float* init, const vfisv_config* cfg,
                         int64_t npix, float* params_out, float* chi2_out, int32_t* iters_out,
                         int32_t* status_out, float* cov_out, void* stream);

/* Companion of vfisv_invert_noalloc (the paper has no counterpart either):
 * synchronise `stream`, then report whether the most recent
 * vfisv_invert_noalloc call on the current device flagged a device error
 * (VFISV_E_DEVICE; the error word is cleared), VFISV_OK if not or if no call
 * was made on this device yet, VFISV_E_CUDA for a CUDA error.  Allocates
 * nothing. */
int vfisv_noalloc_check(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* VFISV_H */
