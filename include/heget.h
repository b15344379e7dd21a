/*
 * heget.h -- C ABI of the GB300-native HEGET hot path.
 *
 * The library evaluates tree-level helicity amplitudes of
 *     u(p1, s1) ubar(p2, s2) -> gamma(k1, l1) ... gamma(kn, ln),   n = 2..8,
 * at many phase-space points at once (Hagiwara et al., arXiv:0908.4403,
 * Sec. 2.1 eqs. (6)-(8)), sums |M|^2 over helicities (Sec. 2.1 eq. (2)),
 * generates flat massless n-body phase space (Sec. 2.1 eq. (4), RAMBO) with
 * the photon cuts of Sec. 2.2 eqs. (9)-(10), and integrates the partonic
 * cross section of Sec. 2.1 eq. (2) by Monte Carlo.
 *
 * Conventions shared by every call:
 *  - Array arguments are DEVICE pointers owned by the caller (for example the
 *    data_ptr() of a torch CUDA tensor) unless a parameter says "host".
 *    The library never frees them and keeps no reference after a call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue work on it and return without waiting, unless
 *    their description says they synchronize.
 *  - Momenta are FP64 GeV, layout [N][n+2][4]: particle order
 *    (p1, p2, k1, ..., kn), components (E, px, py, pz).  p1 is the incoming
 *    u along +z, p2 the incoming ubar along -z.
 *  - Helicity index h in [0, 2^(n+2)): bit0 = s1 (1 -> +1/2, 0 -> -1/2),
 *    bit1 = s2, bit(2+i) = lambda_{i+1} (1 -> +1, 0 -> -1).  A helicity
 *    mask is an array of 2^(n+2)/32 uint32 words (1 word for n <= 3), bit h
 *    of word h/32; NULL selects all 2^(n+2) combinations.
 *  - Generated points are numbered: point i of stream `seed` depends only on
 *    (seed, i).  A call over points i0 .. i0+N-1 needs i0 >= 0 and
 *    i0 + N <= 2^63 - 1, else HEGET_EINVAL.
 *  - Every call returns an int status (HEGET_OK = 0).  On failure,
 *    heget_last_error() returns a message for the calling thread.  No call
 *    aborts, prints, or allocates device memory except heget_create and the
 *    calls documented to grow the context workspace.
 */
#ifndef HEGET_H
#define HEGET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HEGET_OK 0
#define HEGET_EINVAL 1    /* bad argument, or device-side input check failed */
#define HEGET_ENOMEM 2    /* device allocation failed / admission impossible */
#define HEGET_ECUDA 3     /* a CUDA runtime call failed */
#define HEGET_ETIMEOUT 4  /* a bounded wait ran out */
#define HEGET_EBUSY 5     /* no free slot (serving) */
#define HEGET_ENOTFOUND 6 /* unknown ticket (serving) */

/* arithmetic of the spinor / vertex / propagator chain */
#define HEGET_FP32 32
#define HEGET_FP64 64

/* sqrt(s-hat) samplers */
#define HEGET_SAMPLER_FIXED 0   /* sqrt(s-hat) = sqrt_s, boost rapidity y = 0 */
#define HEGET_SAMPLER_UNIFORM 1 /* sqrt(s-hat) uniform in [lo, hi], y = 0 */
#define HEGET_SAMPLER_TOY_PDF 2 /* x1, x2 ~ x^(-1/2)(1-x)^3, sqrt(s-hat) =
                                   2 e_beam sqrt(x1 x2) > floor, y = ln(x1/x2)/2 */

typedef struct heget_ctx heget_ctx;

/* Physics parameters.  alpha: fine-structure constant; q_charge: quark
 * charge in units of e (the couplings gal[0] = gal[1] = -e Q_q of Sec. 4 and
 * Appendix B.3); cuts of Sec. 2.2: photon pT > pt_min, |eta| < eta_max,
 * Delta R > dr_min (dr_min <= 0 disables the Delta R cut).  All cuts strict. */
typedef struct {
    double alpha;
    double q_charge;
    double pt_min;
    double eta_max;
    double dr_min;
} heget_params;

/* sqrt(s-hat) sampler (see HEGET_SAMPLER_*).  max_tries in [1, 64] bounds
 * each rejection loop of the toy PDF; a point whose loops all fail is kept
 * with weight 0 and mask 0. */
typedef struct {
    int kind;
    double sqrt_s;   /* FIXED */
    double lo, hi;   /* UNIFORM */
    double e_beam;   /* TOY_PDF: hadronic sqrt(s) = 2 e_beam */
    double floor;    /* TOY_PDF: accept sqrt(s-hat) > floor */
    int max_tries;   /* TOY_PDF */
} heget_sampler;

/* Monte Carlo result of heget_xsec.  sigma_fb = scale * sum_w / n_total and
 * err_fb = scale * sqrt((<w^2> - <w>^2)/(n_total - 1) ), with scale = 1,
 * or 2 * accept for the toy PDF (q <-> qbar assignment of Sec. 2.1 eq. (1)
 * and the sqrt(s-hat) floor acceptance accept = n_total / n_tries). */
typedef struct {
    double sigma_fb;
    double err_fb;
    double sum_w;     /* compensated sum of per-event weights (fb) */
    double sum_w2;    /* compensated sum of squared weights (fb^2) */
    double accept;
    double reserved;
    int64_t n_pass;   /* events passing the cuts */
    int64_t n_total;  /* events generated (= N) */
    int64_t n_tries;  /* outer sampler attempts (= N unless TOY_PDF) */
    int64_t n_escalated; /* FP32 points recomputed in FP64 */
} heget_xsec_result;

/* Context: binds a CUDA device, holds the physics parameters (defaults:
 * alpha = 1/137.035999, q_charge = 2/3, pt_min = 20, eta_max = 2.5,
 * dr_min = 0.4) and a small workspace.  heget_create allocates the
 * workspace on `device`; returns HEGET_ECUDA if the device is unusable.
 * The workspace (block partials, escalation lists, result staging) is
 * shared by every call on the context: issue them from one host thread at a
 * time and keep them from overlapping on the GPU (one stream per context, or
 * one context per stream).  The request server is the thread-safe way to
 * share a device between submitters. */
int heget_create(int device, heget_ctx** out);
/* Frees the context and its workspace (waits for the batch staging copy);
 * NULL does nothing.  Work still queued on a stream must not use it. */
void heget_destroy(heget_ctx* ctx);
/* Physics parameters of later calls (p: host struct, copied).  EINVAL for a
 * NULL argument, alpha not finite and > 0, q_charge not finite and nonzero,
 * pt_min not finite and >= 0, eta_max not finite and > 0, or dr_min NaN. */
int heget_set_params(heget_ctx* ctx, const heget_params* p);
int heget_get_params(const heget_ctx* ctx, heget_params* p);   /* p: host */
/* The message of the calling thread's last failed call (never NULL; owned by
 * the library, valid until that thread's next call). */
const char* heget_last_error(void);
/* Library name, version and target architecture (static string). */
const char* heget_version(void);

/* Phase space (Sec. 2.1 eq. (4); Sec. 3: random numbers -> phase-space point
 * and Jacobian): for point i in [0, N), draw sqrt(s-hat) with a fixed value,
 * generate n massless photons with RAMBO (Kleiss, Stirling, Ellis 1986) in
 * the partonic CM frame with p1 = (rs/2)(1,0,0,1), p2 = (rs/2)(1,0,0,-1).
 * Random numbers: Philox4x32-10 keyed by `seed`, counter (i lo, i hi,
 * draw / 2, stream), two draws per block, so point i depends only on
 * (seed, i).
 *   momenta: [N][n+2][4] FP64 (may be NULL); weights: [N] FP64 flat
 *   phase-space weight Phi_n(s-hat) in GeV^(2n-4) (may be NULL).
 * EINVAL: n not in [2, 8], N < 0, sqrt_s <= 0. */
int heget_phase_space(heget_ctx* ctx, uint64_t seed, int64_t N, int n,
                      double sqrt_s, double* momenta, double* weights,
                      void* stream);

/* General form: points i0 .. i0+N-1, sampler `smp` (host struct), the cut
 * mask of Sec. 2.2 evaluated with eta_lab = eta_cm + y.  Any output may be
 * NULL.  sqrt_s_out, y_out: [N] FP64; mask_out: [N] uint8 (1 = passes);
 * tries_out: [N] int32 outer sampler attempts.  EINVAL as for
 * heget_phase_space, and for a bad sampler or point range. */
int heget_phase_space_ex(heget_ctx* ctx, uint64_t seed, int64_t i0, int64_t N,
                         int n, const heget_sampler* smp, double* momenta,
                         double* weights, double* sqrt_s_out, double* y_out,
                         uint8_t* mask_out, int32_t* tries_out, void* stream);

/* |M|^2 (Sec. 2.1 eqs. (2), (6)-(8)): for each point,
 *   amp2[i] = sum_{h in hel_mask} |M_h|^2,
 * M_h = sum over the n! photon orderings of the fermion-line chain, including
 * the couplings (-e Q)^n; without colour, spin-average or 1/n! factors.
 * precision: HEGET_FP32 (spinor algebra in FP32, propagator denominators
 * from FP64 invariants) or HEGET_FP64.  momenta: [N][n+2][4]; amp2: [N].
 * The points must conserve momentum, p1 + p2 = sum of the photons (every
 * point of heget_phase_space does, to FP64 rounding): from n = 6 the FP32
 * path forms the denominator of a photon set with more than n/2 photons
 * from its complement, (k_T - p2)^2 = (p1 - k_{all - T})^2.
 * Host-side EINVAL: n not in [2, 8], N < 0, NULL arrays, bad precision.
 * Device-side check: a point with a non-finite entry, or p1 / p2 not
 * massless along +z / -z, gets amp2 = NaN and raises the context's input
 * flag, reported as EINVAL by heget_check (which synchronizes). */
int heget_amp2(heget_ctx* ctx, int n, int64_t N, const double* momenta,
               const uint32_t* hel_mask, int precision, double* amp2,
               void* stream);

/* Gauge (Ward) check of the amplitude (the photon wave functions of Sec. 4
 * are fixed in the light-cone gauge; gauge invariance of the summed
 * orderings is what the validation of Sec. 5 relies on): for each point,
 *   ratio[i] = max_h |M_h(eps*_photon -> k_photon / k_photon^0)| / max_h |M_h|
 * with h over all helicities and the same n! orderings, evaluated in
 * `precision` from the same records as heget_amp2.  For momenta that conserve
 * momentum the numerator vanishes up to rounding, so ratio is ~1e-16 in FP64
 * and ~1e-7 in FP32; a larger value flags broken kinematics or arithmetic.
 * photon in [0, n); momenta [N][n+2][4]; ratio [N] FP64.  Input checks and
 * errors as for heget_amp2 (a bad point gets NaN). */
int heget_ward(heget_ctx* ctx, int n, int64_t N, const double* momenta,
               int photon, int precision, double* ratio, void* stream);

/* The device logarithm of the RAMBO energies q0 = -ln(r r'), Sec. 2.1
 * eq. (4) (Tang's table-driven method, ACM TOMS 16 (1990) 378), exposed so
 * that its accuracy can be checked: y[i] = ln x[i] for N device doubles,
 * each a positive normal number (other inputs give unspecified values).
 * Runs on the current device; EINVAL for N < 0 or NULL arrays. */
int heget_log_table(const double* x, double* y, int64_t N, void* stream);

/* The device cosine and sine of the RAMBO azimuth phi = 2 pi r, Sec. 2.1
 * eq. (4), exposed so that their accuracy can be checked.  words [N][2]
 * (device uint32: lo, hi) are the two random words of one uniform,
 * r = (2m + 1) 2^-53 with m = ((hi << 32) | lo) >> 12 (the generator's layout);
 * cs [N][2] (device doubles) receives (cos phi, sin phi).  Runs on the
 * current device; EINVAL for N < 0 or NULL arrays. */
int heget_sincos_2pi(const uint32_t* words, double* cs, int64_t N, void* stream);

/* The device double -> float conversion of the FP32 point records (round to
 * nearest even by integer operations; results below the normal float range
 * become signed zeros), exposed so that it can be checked against the
 * hardware conversion: y[i] = (float) x[i] for N device values.  Runs on the
 * current device; EINVAL for N < 0 or NULL arrays. */
int heget_f32_round(const double* x, float* y, int64_t N, void* stream);

/* Synchronizes `stream` and reports (then clears) the device-side input
 * flag raised by heget_amp2 / heget_ward: HEGET_EINVAL if set. */
int heget_check(heget_ctx* ctx, void* stream);

/* Monte Carlo partonic cross section (Sec. 2.1 eq. (2); summation of
 * Sec. 3.1 step 5) over points i0 .. i0+N-1: per event
 *   w = (1/2s)(1/2^2)(1/3^2) 3 sum_h |M_h|^2 (1/n!) Phi_n(s) mask  [fb],
 * accumulated in compensated FP64 (double-double per thread, then a
 * fixed-order tree), so the result is deterministic for fixed arguments.
 * result_dev: device array of sizeof(heget_xsec_result) bytes receiving the
 * result; w_out (optional, may be NULL): [N] per-event weights.  Uses the
 * context workspace (grown on demand; not thread-safe per context).
 * Enqueues only. */
int heget_xsec_async(heget_ctx* ctx, int n, uint64_t seed, int64_t i0,
                     int64_t N, const heget_sampler* smp, int precision,
                     heget_xsec_result* result_dev, double* w_out,
                     void* stream);

/* heget_xsec_async over points 0 .. N-1, then copies the result to the host
 * struct `out` and synchronizes `stream`. */
int heget_xsec(heget_ctx* ctx, int n, int64_t N, uint64_t seed,
               const heget_sampler* smp, int precision,
               heget_xsec_result* out, void* stream);

/* One request of a mixed-n batch (heget_xsec_batch): points i0 .. i0+N-1 of
 * stream `seed` for n photons at `precision` with sampler `sampler`;
 * result_dev (device, sizeof(heget_xsec_result) bytes) receives the result,
 * w_out (device, optional) the N per-event weights. */
typedef struct {
    int n;
    int precision;
    uint64_t seed;
    int64_t i0;
    int64_t N;
    heget_sampler sampler;
    heget_xsec_result* result_dev;
    double* w_out;
} heget_xsec_request;

/* Many cross sections in one fused launch per precision (batching of the
 * serving path; the paper runs one process per kernel call, Sec. 3.1).
 * Every request is cut into point tiles: the context's xsec tile if set
 * (heget_set_tile), else with the tree the tiles heget_xsec uses on the
 * plain (non-warp-specialised) path, with the subset recursion tiles of 128
 * points (FP32: 64 from n = 5; FP64: 64 at n = 4, 16 at
 * n = 5, 8 from n = 6), the largest that let two blocks share an SM.  The
 * kernel is compiled once per algorithm.  The tiles of all requests, whatever
 * their n and N, form one work list that a single kernel walks, and each
 * request's tile partials are combined in tile order, so a request's result
 * does not depend on what else is in the batch.  reqs: host array of `count`
 * requests.  At most 2^22 tiles per precision and call (HEGET_EINVAL
 * beyond: split the batch).  Grows the context workspace on demand, and
 * synchronizes `stream` before returning. */
int heget_xsec_batch(heget_ctx* ctx, const heget_xsec_request* reqs, int count,
                     void* stream);

/* Kinematic distributions (Sec. 5, Fig. 2: the largest photon transverse
 * momentum and the photons' Delta R separations).  Observables, in GeV for
 * momenta, with pT = sqrt(px^2 + py^2), the lab pseudorapidity
 * eta = asinh(pz / pT) + y (y the boost rapidity of the toy-PDF sampler, 0
 * otherwise, as for the cuts of Sec. 2.2), phi = atan2(py, px) and
 * Delta R = sqrt(Delta eta^2 + Delta phi^2) with Delta phi in [0, pi]. */
#define HEGET_OBS_PT_MAX 0 /* largest photon pT of the event: 1 entry */
#define HEGET_OBS_PT 1     /* pT of each photon: n entries */
#define HEGET_OBS_ETA 2    /* eta of each photon: n entries */
#define HEGET_OBS_DR 3     /* Delta R of each photon pair: n(n-1)/2 entries */
#define HEGET_OBS_DR_MIN 4 /* smallest Delta R of the event: 1 entry */
#define HEGET_OBS_SQRT_S 5 /* sqrt(s-hat): 1 entry */

/* One histogram: `nbins` uniform bins on [lo, hi), closed on the left, plus
 * an underflow bin (x < lo, and NaN) and an overflow bin (x >= hi).  x falls
 * in bin 1 + floor((x - lo) * (nbins / (hi - lo))), evaluated in FP64. */
typedef struct {
    int32_t observable; /* HEGET_OBS_* */
    int32_t nbins;      /* >= 1 */
    double lo, hi;      /* finite, lo < hi, nbins / (hi - lo) finite */
} heget_hist_spec;

#define HEGET_HIST_MAX_SPECS 8
#define HEGET_HIST_MAX_BINS 1024 /* sum over the specs of nbins + 2 */

/* Weighted histograms of the events (seed, i0 .. i0+N-1) of n photons: each
 * entry of an event adds its weight w[j] to its bin's sum of weights and w[j]^2
 * to its sum of squares.  The events are those of heget_xsec and
 * heget_phase_space_ex with the same (n, seed, i0, N, sampler) and the
 * context's parameters; their momenta are regenerated on the device, so w
 * is typically the w_out of a heget_xsec_async call on the same points
 * (0 for the points that fail the cuts).
 * w: N device doubles.  specs: host array of 1 <= nspec <= HEGET_HIST_MAX_SPECS
 * histograms with at most HEGET_HIST_MAX_BINS bins in all.  out: device
 * doubles, for each spec in order its nbins + 2 bins (underflow, the bins,
 * overflow), each as (sum w, sum w^2): 2 sum (nbins + 2) values, written
 * (zeros for N = 0).  Each block sums its tiles' entries per bin in a fixed
 * order and folds the tile sums into double-double sums, combined in block
 * order: results are reproducible bit for bit on a given GPU model (the
 * grid is one resident wave).  EINVAL for bad specs, n, N, sampler or NULL
 * arrays (N > 0). */
int heget_hist(heget_ctx* ctx, int n, uint64_t seed, int64_t i0, int64_t N,
               const heget_sampler* sampler, const double* w,
               const heget_hist_spec* specs, int nspec, double* out,
               void* stream);

/* heget_xsec_async in two halves: heget_xsec_launch enqueues only the fused
 * event kernel, leaving its block partials in the context workspace;
 * heget_xsec_finalize enqueues the fixed-order combination of the partials of
 * the most recent heget_xsec_launch on this context into result_dev.  The
 * pair is equivalent to heget_xsec_async and exists so that callers can time
 * or graph-capture the halves separately.  Errors as for heget_xsec_async;
 * heget_xsec_finalize also refuses a NULL result_dev. */
int heget_xsec_launch(heget_ctx* ctx, int n, uint64_t seed, int64_t i0,
                      int64_t N, const heget_sampler* smp, int precision,
                      double* w_out, void* stream);
int heget_xsec_finalize(heget_ctx* ctx, heget_xsec_result* result_dev,
                        void* stream);

/* Ordering-sum algorithm of a context (amp2, xsec, batch, graphs, server).
 *  HEGET_ALG_TREE (default): the paper's method -- every ordering of the
 *    photons along the fermion line (Sec. 2.1 eqs. (6)-(8), the permutation
 *    program of Appendix A.2), each shared ordered prefix computed once, and
 *    for n >= 4 each pair of last photons closed against per-point currents
 *    from the u end (sub-current reuse from both ends).
 *  HEGET_ALG_SUBSET: the same sum regrouped by the SET of photons attached so
 *    far (a step's propagator depends on the set, not the order), so that the
 *    current of each set and helicity assignment is computed once:
 *    sum_k C(n,k) k 2^k chain steps per point instead of
 *    2^n sum_l n!/(n-l)!.  Not in the paper; same |M|^2 up to rounding.
 * heget_ward and heget_xsec_noalloc always use the tree.  EINVAL for an
 * unknown algorithm; heget_get_algorithm returns -1 for a NULL context. */
#define HEGET_ALG_TREE 0
#define HEGET_ALG_SUBSET 1
int heget_set_algorithm(heget_ctx* ctx, int alg);
int heget_get_algorithm(const heget_ctx* ctx);

/* Helicity sampling (off by default).  The paper's events each carry one
 * random helicity combination (Sec. 3, program step 4); with sampling on,
 * the cross-section paths of a context (heget_xsec*, batch, graphs, server)
 * do the same: point i draws h = floor(2^(n+2) u), u draw 0 of generator
 * stream 2 (key = seed, counter = (i lo, i hi, 0, 2)), and its weight uses
 * 2^(n+2) |M_h|^2 instead of the sum over all helicities; h with
 * sigma1 = sigma2 gives weight 0.  The estimate has the same mean and a
 * larger variance, at the same cost (the kernels evaluate every helicity of
 * a point together).  heget_amp2, heget_ward and heget_xsec_noalloc are
 * unaffected.  EINVAL for a NULL context or on not 0/1; the getter returns -1
 * for a NULL context. */
int heget_set_helicity_sampling(heget_ctx* ctx, int on);
int heget_get_helicity_sampling(const heget_ctx* ctx);

/* FP32 -> FP64 escalation (the FP32 precision policy: FP32 where it is
 * accurate, FP64 where it is not).  In FP32, heget_amp2 and the fused cross
 * section (heget_xsec, heget_xsec_async, heget_xsec_launch, graphs) bound
 * each point's rounding error: with B_h >= sum over orderings |A_pi,h| from
 * norm bounds of the chain steps, the relative error of sum_h w_h |A_h|^2 is
 * at most about u32 sqrt(sum_h w_h B_h^2 / sum_h w_h |A_h|^2), u32 = 2^-24.
 * Points whose bound exceeds tau are recomputed in FP64 by a second kernel
 * on the same stream (with the subset recursion, whatever the context's
 * algorithm: the same |M|^2 up to rounding, far cheaper at large n):
 * heget_amp2 overwrites their |M|^2, the cross section replaces their FP32
 * weights by the FP64 ones (in w_out too) and counts them in n_escalated.
 * tau = 0 (the default) turns it off; 1e-4 is the threshold of the FP32
 * accuracy target (the bound is conservative: at n = 8 it flags a few per
 * cent of points whose actual FP32 error is far below tau, and their FP64
 * recomputation is the cost).  Batches, the server and heget_xsec_noalloc do
 * not escalate (their n_escalated is 0), nor does a heget_amp2 call of more
 * than 2^31 - 1 points (its row list is indexed in int32).
 * heget_amp2_escalated synchronizes `stream` and returns the number of rows
 * the last FP32 heget_amp2 on ctx recomputed. */
int heget_set_escalation(heget_ctx* ctx, double tau);
int heget_get_escalation(const heget_ctx* ctx, double* tau);
int heget_amp2_escalated(heget_ctx* ctx, void* stream, int64_t* count);

/* Launch shape (this library's knob; the paper's analogue is the register /
 * block-size scan of Sec. 6.1): points per block tile used by heget_amp2
 * (kind 0) or heget_xsec* (kind 1) for n photons at `precision`.  tile = 0
 * restores the default (for heget_amp2 with the subset recursion, larger
 * tiles than the tree's: 128 points at n = 4, 5 in FP32, 64 at n = 6, 32 at
 * n = 7, 8); otherwise tile must be a positive multiple of
 * 256 / 2^n and at most 4096.  A tile whose shared memory exceeds the device
 * limit makes the next launch fail with HEGET_ECUDA. */
int heget_set_tile(heget_ctx* ctx, int n, int precision, int kind, int tile);
int heget_get_tile(const heget_ctx* ctx, int n, int precision, int kind);

/* CUDA graphs for the mixed-n launches (A9): with on = 1, heget_xsec_batch
 * and servers started afterwards on this context launch each precision's
 * work-list kernel and finalisation as a CUDA graph per launch-shape bucket
 * (the same item and request counts, grid and shared memory), captured on
 * first use and replayed when the bucket recurs; the results are the same
 * bits as direct launches.  At most 32 buckets are kept (the oldest goes
 * first); growing the batch workspace drops them.  heget_get_graphs returns
 * the setting (-1 for a NULL context) and the numbers of captures and
 * replays so far (either pointer may be NULL).  EINVAL for a NULL context or
 * `on` not 0/1. */
int heget_set_graphs(heget_ctx* ctx, int on);
int heget_get_graphs(const heget_ctx* ctx, int64_t* captures, int64_t* replays);

/* Tile-kernel shape of the fused cross section (heget_xsec*, graphs) for n
 * photons at `precision`: 0 (the default: the warp-specialised kernel where it
 * applies, else the tile kernel's default shape) or, for the FP32 tree at
 * n = 6..8, shapes 1..3 -- tile kernels of other thread counts, helicity
 * configurations per lane (rows) and subtree groups (the launch-shape knobs of
 * the paper's Sec. 6.1 scan, as far as they exist on this design).
 * heget_shape_info reports a shape's threads per block, rows per lane and
 * groups (all 0 for shape 0).  Shapes apply to the prefix tree; the subset
 * recursion and FP32 escalation run shape 0.  EINVAL for a NULL context, bad
 * n or precision, or a shape that does not exist there; heget_get_shape
 * returns -1 for bad arguments. */
int heget_set_shape(heget_ctx* ctx, int n, int precision, int shape);
int heget_get_shape(const heget_ctx* ctx, int n, int precision);
int heget_shape_info(int n, int precision, int shape, int* threads,
                     int* rows_per_lane, int* groups);

/* Autotuner (this library's; the paper scans registers x block size by hand,
 * Sec. 6.1 / Fig. 3): times heget_amp2 (kind 0) or heget_xsec (kind 1) for
 * n photons at `precision` on `probe_points` synthetic points for every
 * candidate launch -- for kind 1 every shape (heget_set_shape) with its
 * default tile and the tiles 256/2^n x 2^k up to 1024; for kind 0 the tiles
 * -- keeps the fastest in the context and returns it (*best_tile, 0 =
 * default; *best_shape, may be NULL) with its time (*best_ms).  Allocates and
 * frees temporary probe buffers; synchronizes.  heget_autotune_save /
 * heget_autotune_load store and restore the context's tuned tiles and shapes
 * in a text file keyed by GPU name (other GPUs' lines are kept).  EINVAL for
 * bad n, precision, kind, probe_points < 1 or a path that cannot be opened;
 * ECUDA if no candidate ran (the context keeps its previous tile and shape). */
int heget_autotune(heget_ctx* ctx, int n, int precision, int kind,
                   int64_t probe_points, int* best_tile, double* best_ms);
int heget_autotune_shape(heget_ctx* ctx, int n, int precision,
                         int64_t probe_points, int* best_shape, int* best_tile,
                         double* best_ms);
int heget_autotune_save(const heget_ctx* ctx, const char* path);
int heget_autotune_load(heget_ctx* ctx, const char* path);

/* CUDA graph of one cross-section step: heget_xsec_launch +
 * heget_xsec_finalize for n, N, sampler and precision as given, captured
 * once; heget_graph_launch replays it for a new (seed, i0) by updating the
 * captured event kernel's arguments.  result_dev receives each replay's
 * result.  A graph uses its context's workspace: replays of graphs of one
 * context must be ordered on one stream.  heget_graph_xsec: EINVAL for a
 * NULL out or result_dev, N < 1, or a bad n, precision or sampler (the
 * escalation lists are grown before capture, since a capture cannot
 * allocate); ECUDA if capture or instantiation fails.  heget_graph_launch:
 * EINVAL for a NULL graph or i0 outside the point-range rule; ECUDA if the
 * update or the launch fails.  heget_graph_destroy(NULL) does nothing. */
typedef struct heget_graph heget_graph;
int heget_graph_xsec(heget_ctx* ctx, int n, int64_t N, const heget_sampler* smp,
                     int precision, heget_xsec_result* result_dev,
                     heget_graph** out);
int heget_graph_launch(heget_graph* g, uint64_t seed, int64_t i0, void* stream);
void heget_graph_destroy(heget_graph* g);

/* Request server (continuous batching).  The paper has no counterpart: it
 * runs one cross section per process (Sec. 3.1); this is a service of this
 * library for many concurrent cross-section requests of mixed n.
 *
 * heget_server_start starts a worker thread that owns one stream on ctx's
 * device.  Submitted requests wait in arrival order until fewer than
 * max_inflight are admitted and the device arena (arena_bytes, default
 * min(256 MiB, free HBM x (1 - hbm_reserve_frac))) has room for their tile
 * partials (64 bytes per tile of heget_xsec_batch's tile size, plus the
 * result).  Each launch of the mixed-n batch kernel takes tiles round-robin
 * from every admitted request until about max_launch_work FP32-flop
 * equivalents are filled (the amplitude flops of the server's algorithm per
 * point, plus the event generation) and at least
 * two tiles per SM are taken (when the admitted requests have them), so requests
 * arriving while others run share the next launch with them; up to two
 * launches are in flight.  A request's result is bitwise the
 * heget_xsec_batch result of the same request, whatever else shared its
 * launches.  Zero fields of cfg (or cfg = NULL) take the defaults:
 * max_inflight 256, max_launch_work 2e11, hbm_reserve_frac 0.1.  The server
 * keeps the ordering-sum algorithm ctx has at heget_server_start.  ctx must
 * outlive the server and must not change its parameters or tiles while
 * requests are in flight. */
typedef struct heget_server heget_server;
typedef struct {
    int max_inflight;        /* admitted requests at once (>= 1) */
    double max_launch_work;  /* FP32-flop equivalents per launch */
    double hbm_reserve_frac; /* share of free HBM the arena leaves alone */
    uint64_t arena_bytes;    /* device arena size; 0 = default */
} heget_server_cfg;

/* One request: points i0 .. i0+N-1 (N >= 1) of stream `seed`, n photons at
 * `precision` with `sampler`, as for heget_xsec_async. */
typedef struct {
    int n;
    int precision;
    uint64_t seed;
    int64_t i0;
    int64_t N;
    heget_sampler sampler;
} heget_request;

/* A finished request: status HEGET_OK with `result`, HEGET_ECUDA if a launch
 * failed (the server then stops taking work), HEGET_EBUSY if the server
 * stopped before the request was admitted.  Times are seconds on a
 * monotonic host clock: submission, admission, result available on host. */
typedef struct {
    heget_xsec_result result;
    double t_submit, t_admit, t_done;
    int status;
    int reserved;
} heget_result;

int heget_server_start(heget_ctx* ctx, const heget_server_cfg* cfg,
                       heget_server** out);
/* Queues a request (host struct, copied) and returns its ticket.  Fails with
 * HEGET_EINVAL on a bad request, HEGET_ENOMEM if it could never fit in the
 * arena, HEGET_EBUSY once the server is stopping.  Thread-safe. */
int heget_submit(heget_server* s, const heget_request* q, uint64_t* ticket);
/* HEGET_OK and *out if the request is finished (the ticket is then
 * released), HEGET_EBUSY if not yet, HEGET_ENOTFOUND for an unknown or
 * already released ticket.  Never blocks. */
int heget_poll(heget_server* s, uint64_t ticket, heget_result* out);
/* As heget_poll, but waits up to timeout_s seconds (>= 0, else
 * HEGET_EINVAL; capped at 1e7 s); HEGET_ETIMEOUT if the request is still
 * running then (the ticket stays valid). */
int heget_wait(heget_server* s, uint64_t ticket, double timeout_s,
               heget_result* out);
/* Cancels requests not yet admitted (they finish with HEGET_EBUSY), lets
 * admitted ones run to completion, joins the worker and frees everything;
 * unclaimed results are dropped.  Returns HEGET_ECUDA if a launch failed. */
int heget_server_stop(heget_server* s);

/* Device FMA throughput: runs independent FMA chains (8 per thread) in
 * every thread of a grid that fills the GPU and reports the achieved rate in
 * TFLOP/s (2 flops per FMA) in *tflops.  precision: HEGET_FP32 or HEGET_FP64.
 * The measured denominator of the FMA-pipe roofline.  Uses the legacy
 * default stream and a temporary device buffer; synchronizes.  EINVAL for a
 * NULL argument or a bad precision; ECUDA if a launch fails. */
int heget_measure_fma_peak(heget_ctx* ctx, int precision, double* tflops);

/* heget_xsec_async for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a service of this library.  Such callers
 * include applications whose device memory is owned by a framework arena or
 * a custom allocator that a library must not bypass, and latency-critical
 * paths that cannot afford the implicit synchronisation of cudaMalloc.
 *
 * No context is needed and nothing is allocated: no cudaMalloc, no cudaFree,
 * no allocating library routine.  The per-block partial sums that
 * heget_xsec_async keeps in the context workspace live here in a static
 * array of 4096 entries (256 KiB) that every GPU loading the library holds
 * until the process exits.  The caller passes the inputs and result_dev
 * (device array of sizeof(heget_xsec_result) bytes) as for
 * heget_xsec_async; params (host, may be NULL for the defaults) replaces the
 * context's parameters; `device` selects the GPU.
 *
 * It launches what heget_xsec_async launches by default (prefix tree), so
 * the results are the same bits.  Limit: a call needs one partial per block
 * of its launch; if that exceeds 4096 the call fails with HEGET_EINVAL and a
 * message giving the largest N for this n and precision.  FP32 at n <= 5
 * launches one resident wave of blocks and has no limit; otherwise N may be
 * at most 4096 x the default xsec tile (for example 262,144 points at n = 6,
 * 131,072 at n = 7 and 32,768 at n = 8 in FP32, 524,288 at n <= 4 in FP64).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it with the CUDA context current at the
 * time; make that first call before any stream capture.  A call under
 * another context of that device (after cudaDeviceReset, or a context made
 * current through the driver API) looks the address up again, so the same
 * rule holds for the first call under each new context.
 * Every call shares the one array per device and leaves its contents
 * behind; nothing in it needs clearing, but calls that overlap on the GPU
 * (concurrent streams) race on it and must not be issued.
 * EINVAL, as heget_xsec_async: bad n, N < 0, i0 < 0 or i0 + N beyond int64,
 * bad precision or sampler, NULL result_dev, params that heget_set_params
 * refuses, a device that is not present, or N beyond the limit above. */
int heget_xsec_noalloc(int device, int n, uint64_t seed, int64_t i0, int64_t N,
                       const heget_sampler* smp, const heget_params* params,
                       int precision, heget_xsec_result* result_dev,
                       void* stream);

/* Compensated sums of x[0..N-1] (the accumulator of heget_xsec, exposed):
 * out_dev[0] = sum x, out_dev[1] = sum x^2, each rounded once from a
 * double-double accumulation in a fixed order (the same bits for the same
 * x on a given GPU model).  x: [N] device doubles; out_dev: 2 device doubles.  Uses
 * the context workspace.  EINVAL for a NULL context or out_dev, N < 0, or
 * x NULL with N > 0. */
int heget_sum(heget_ctx* ctx, const double* x, int64_t N, double* out_dev,
              void* stream);

/* Combination of the results of disjoint point shards, on the host (the
 * summation step of the paper's program, Sec. 3.1, spread over processes;
 * no GPU needed).  heget_xsec_combine: parts[0 .. nparts-1] (host structs,
 * in the order given) are merged as if one call had processed all their
 * points: sum_w and sum_w2 each accumulated as a double-double in that order
 * and rounded once, counts added, and sigma, its error and the acceptance
 * recomputed with the formulas of heget_xsec (Sec. 2.1 eq. (1)-(2): for the
 * toy PDF, sampler_kind HEGET_SAMPLER_TOY_PDF, the factor 2 of the q <-> qbar
 * assignment times the acceptance of the sqrt(s-hat) floor).
 * heget_hist_combine: len-element arrays parts[0 .. nparts-1] (host, e.g.
 * heget_hist outputs copied back) added element by element with TwoSum in
 * that order and rounded once into out (host, len doubles; it may be one of
 * the parts).  Same bits for the same parts in the same order.  EINVAL for
 * nparts < 0, len < 0, a NULL out, parts NULL with nparts > 0, or an unknown
 * sampler kind. */
int heget_xsec_combine(const heget_xsec_result* parts, int nparts,
                       int sampler_kind, heget_xsec_result* out);
int heget_hist_combine(const double* const* parts, int nparts, int64_t len,
                       double* out);

#ifdef __cplusplus
}
#endif
#endif /* HEGET_H */
