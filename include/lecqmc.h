/*
 * lecqmc.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * linear canonical-ensemble QMC (LEC-QMC, Hong, Chen, Xu, arXiv 2601.08552).
 *
 * The library runs Markov chains of the canonical-ensemble determinant QMC of
 * the Hubbard model H = sum_ij K_ij c^dag_i c_j + U sum_i n_iup n_idn
 * (Eq. 5) at fixed N_up and N_dn.  A configuration is a pair (eta, s): a Fock
 * state (ordered occupied sites per spin, the columns of P_eta) and discrete
 * Hubbard-Stratonovich fields s[slice][site] = +-1.  Its weight is
 * prod_sigma det[P^T B_sigma(beta,0) P] (Eq. 1) with
 * B(beta,0) = B_{L-1} ... B_0 and B_l = e^{-dtau K} e^{-dtau V(s_l)}.
 * A sweep is: field updates over all slices upward, N_up then N_dn
 * particle-hole swaps by the stabilized QR update (removal by Givens
 * rotations, addition by propagating one column and orthogonalising it, SM
 * Sec. I), then field updates downward with measurements at the
 * stabilization boundaries.  Cost O(beta N N_e^2) per sweep.
 *
 * Conventions
 *  - Every call returns lq_status; nothing throws or exits across the ABI.
 *    lq_last_error() gives a thread-local message for the last failure.
 *  - Pointers named host_* or documented as host arrays are caller-owned host
 *    memory; the library copies them.  The library owns its device memory.
 *  - Handles are not thread-safe: use one handle per thread.
 *  - Work is queued on the CUDA stream given at creation; calls that return
 *    data to the host synchronize that stream first.  lq_sim_sync() reports
 *    deferred device errors (LQ_ENUMERIC for a singular overlap, a CholeskyQR
 *    breakdown or a non-finite ratio).
 *  - Indices are 0-based: slices 0..L-1 (L = round(beta/dtau)), sites
 *    0..N-1, spin 0 = up, 1 = down.
 */
#ifndef LECQMC_H
#define LECQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LQ_OK = 0,
  LQ_EINVAL = 1,      /* bad argument (range, size, null) */
  LQ_ENOMEM = 2,      /* device or host allocation failed */
  LQ_ECUDA = 3,       /* a CUDA runtime call failed */
  LQ_ENUMERIC = 4,    /* singular overlap, QR breakdown or non-finite ratio */
  LQ_ETIMEOUT = 5,    /* a bounded device wait gave up */
  LQ_EBUSY = 6,       /* a queue is full */
  LQ_ENOTFOUND = 7,   /* no such request / result not ready */
  LQ_EUNSUPPORTED = 8 /* a size outside what the library supports */
} lq_status;

/* precision modes.
 * LQ_FP64: everything in FP64.
 * LQ_MIXED: the N x N_sigma panels (storage and slice propagation) in FP32;
 *   QR, log-det factors, the N_sigma x N_sigma inverses, field-flip algebra and
 *   all Metropolis ratios in FP64.
 * LQ_MIXED_DW: as LQ_MIXED, but the per-site field-flip algebra (the
 *   Sherman-Morrison ratio and rank-1 update of the inverse) runs in
 *   double-word FP32 arithmetic (pairs of floats, about 2^-46 relative per
 *   operation) instead of FP64, whose per-instruction cost on GB300 makes the
 *   sequential flip loop latency bound. */
#define LQ_FP64 0
#define LQ_MIXED 1
#define LQ_MIXED_DW 2

/* observables of one sweep record: the mean over the measurements of the
 * sweep of sign * O (index 0 is the sign itself). */
#define LQ_NOBS 9
#define LQ_OBS_SIGN 0
#define LQ_OBS_NUP 1   /* sum_i <n_i,up> (= N_up, an invariant) */
#define LQ_OBS_NDN 2
#define LQ_OBS_DOCC 3  /* (1/N) sum_i <n_i,up n_i,dn> */
#define LQ_OBS_EKIN 4  /* (1/N) sum_sigma sum_ij K_ij <c^dag_i c_j> */
#define LQ_OBS_SZZ00 5 /* <S^z_A S^z_A> / (N/2), sublattice label 0 */
#define LQ_OBS_SZZ11 6
#define LQ_OBS_SZZ01 7
#define LQ_OBS_SPAR 8  /* S^par(q=0) = (1/(N/2)) sum_ij <S^x_i S^x_j + S^y_i S^y_j> */

/* largest particle number per spin the library supports */
#define LQ_MAX_PARTICLES 512

typedef struct lq_lattice lq_lattice;
typedef struct lq_sim lq_sim;

/* ---- lattices (the hopping matrix K; Eq. 5 and SM Sec. III) ------------ */

/* K from bonds: K_ij = K_ji = kij[b] for b = (bi[b], bj[b]), plus an optional
 * onsite term onsite[i] (K_ii) and an optional sublattice label 0/1 per site
 * (default i % 2).  The bond order fixes the checkerboard: each bond goes to
 * the lowest family in which neither of its sites is used yet, and
 * e^{-dtau K} is applied as E_{G-1} ... E_0 C_eps with E_g the exact product
 * of the 2x2 bond exponentials of family g and C_eps = diag(e^{-dtau K_ii}).
 * All arrays are host arrays of n_bonds (or n_sites) entries; copied.
 * Errors: LQ_EINVAL for n_sites < 1, a site out of range, i == j. */
lq_status lq_lattice_from_bonds(int32_t n_sites, int32_t n_bonds, const int32_t* bi, const int32_t* bj,
                                const double* kij, const double* onsite, const int32_t* sublattice,
                                lq_lattice** out);
/* 1D chain, K = -t on (i, i+1): bonds with even i, then odd i (periodic wrap
 * in the odd group). Sublattice i % 2. */
lq_status lq_lattice_chain(int32_t n_sites, double t, int32_t periodic, lq_lattice** out);
/* Lx x Ly square lattice, site x + Lx*y, K = -t: x-bonds with even x, odd x,
 * y-bonds with even y, odd y.  Sublattice (x + y) % 2. */
lq_status lq_lattice_square(int32_t lx, int32_t ly, double t, int32_t periodic, lq_lattice** out);
/* One-dimensional BCL flat-band model, H_eff(k) = S(k) S(k)^dag with
 * S1 = t1 + t2 e^{-ik}, S2 = t3 + t4 e^{-ik} (SM Sec. III): sites
 * A1_R = 2R, A2_R = 2R+1; onsite t1^2+t2^2 (A1), t3^2+t4^2 (A2); hoppings
 * A1_R-A1_{R+1} t1 t2, A2_R-A2_{R+1} t3 t4, A1_R-A2_R t1 t3 + t2 t4,
 * A1_R-A2_{R+1} t1 t4, A1_R-A2_{R-1} t2 t3.  The lowest band is exactly flat
 * at 0.  Sublattice A1 = 0, A2 = 1. */
lq_status lq_lattice_flatband(int32_t n_cells, double t1, double t2, double t3, double t4, int32_t periodic,
                              lq_lattice** out);
/* Two-leg cross-stitch ladder: rung -t_intra, legs -t_leg, crossings
 * a_R-b_{R+1}, b_R-a_{R+1} of -t_cross (flat band at +t_intra). */
lq_status lq_lattice_cross_stitch(int32_t n_cells, double t_intra, double t_leg, double t_cross, int32_t periodic,
                                  lq_lattice** out);
/* sizes: sites, bonds, checkerboard families */
lq_status lq_lattice_info(const lq_lattice* lat, int32_t* n_sites, int32_t* n_bonds, int32_t* n_families);
/* the bond list in build order with each bond's family (host arrays of n_bonds) */
lq_status lq_lattice_bonds(const lq_lattice* lat, int32_t* bi, int32_t* bj, double* kij, int32_t* family);
lq_status lq_lattice_destroy(lq_lattice* lat);

/* ---- simulations -------------------------------------------------------- */

typedef struct {
  double U;        /* Hubbard U: U > 0 spin-channel HS, U < 0 charge channel */
  double beta;     /* inverse temperature */
  double dtau;     /* Trotter step; L = round(beta/dtau) must be within 1e-9 */
  int32_t n_up, n_dn;
  int32_t n_stab;  /* tau_w: slices between QR restabilizations */
  int32_t precision; /* LQ_FP64, LQ_MIXED or LQ_MIXED_DW */
  uint64_t seed;   /* Philox4x32-10 key */
  int32_t swap_mode; /* Fock-swap target: LQ_SWAP_UNIFORM or LQ_SWAP_NEIGHBOUR (0 = uniform) */
  int32_t left_swaps; /* 0: Fock swaps at tau = beta only, after the up pass (default).  1: also a
                       * second set of N_up + N_dn attempts at tau = 0 after the down pass, walking
                       * the left chain (the right chain of the transposed propagator
                       * B(beta,0)^T, whose weight det[P^T B^T P] is the same).  Other values:
                       * LQ_EINVAL. */
  int32_t kinetic;    /* how e^{-dtau K} of B_l = e^{-dtau K} e^{-dtau V(s_l)} (Eq. 1) is applied:
                       * LQ_CHECKERBOARD (0, default) or LQ_EXACT (1); other values LQ_EINVAL */
} lq_params;

/* Kinetic propagator.  The paper's linear scaling needs e^{-dtau K} applied in
 * O(N) per panel column; it does not say how.
 * LQ_CHECKERBOARD: B_K = E_{G-1} ... E_0 C_eps, each E_g the exact product of
 *   the 2x2 bond exponentials of checkerboard family g, C_eps = diag(e^{-dtau
 *   K_ii}).  Exact for its own Trotter splitting; G passes over the bonds.
 * LQ_EXACT: B_K = e^{-dtau K} itself (no splitting error), applied as the
 *   Taylor polynomial of degree q in the sparse -dtau K, q the smallest degree
 *   whose remainder is below 1e-17 relative (about 10-20 for dtau = 0.05):
 *   q sparse products per slice, still O(N N_sigma) per slice.  Needs
 *   theta = dtau max_i sum_j |K_ij| <= 2 (LQ_EUNSUPPORTED otherwise) and a
 *   shared-memory staging buffer of two panel columns. */
#define LQ_CHECKERBOARD 0
#define LQ_EXACT 1

/* Fock-swap proposals.  A swap removes the particle of a uniformly drawn
 * occupied column k and adds one at a target site j.  UNIFORM draws j
 * uniformly among the empty sites.  NEIGHBOUR draws j uniformly among the
 * empty nearest neighbours E(i) of the removed particle's site i (distinct
 * bond partners; no move if there is none) and accepts with the
 * Metropolis-Hastings factor |E(i)| / |E'(j)|, E'(j) being the empty
 * neighbours of j after the move.  The paper fixes the weight ratio of a
 * Fock-state move, not its proposal law. */
#define LQ_SWAP_UNIFORM 0
#define LQ_SWAP_NEIGHBOUR 1

/* optional device allocator (e.g. a framework's caching allocator); stream is
 * the cudaStream_t the memory is used on.  NULL -> cudaMalloc/cudaFree. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
} lq_allocator;

/* Create n_chains independent chains.  lattices[c] and params[c] describe
 * chain c (sizes may differ between chains; all chains share one precision).
 * chain_ids (nullable) gives the Philox chain word of each chain (default c).
 * cuda_stream is a cudaStream_t (NULL = default stream).  Fields start at +1
 * and occupations at the first N_sigma sites until lq_sim_init or the setters
 * run.  Errors: LQ_EINVAL (a parameter out of range),
 * LQ_EUNSUPPORTED (n_up or n_dn > LQ_MAX_PARTICLES), LQ_ENOMEM. */
lq_status lq_sim_create(const lq_lattice* const* lattices, const lq_params* params, int32_t n_chains,
                        const uint32_t* chain_ids, void* cuda_stream, const lq_allocator* alloc, lq_sim** out);
/* Draw fields (uniform +-1) and Fock states (Fisher-Yates, sorted) from each
 * chain's seed on the device, then build the right and left QR chains
 * (B_i Q_{i-1} = Q_i V_i, SM Sec. I.A).  Asynchronous. */
lq_status lq_sim_init(lq_sim* sim);
/* Hubbard-Stratonovich fields s of Eq. 1 for one chain from a host array
 * (L x N, row = slice, values +-1); rebuilds that chain's QR chains.
 * Errors: LQ_EINVAL for a value != +-1. */
lq_status lq_sim_set_fields(lq_sim* sim, int32_t chain, const int8_t* host_s);
lq_status lq_sim_get_fields(lq_sim* sim, int32_t chain, int8_t* host_s);
/* The Fock state eta of Eq. 1: ordered occupied sites (the columns of P_eta)
 * of one chain; rebuilds its chains.  Errors: LQ_EINVAL for a repeated or
 * out-of-range site. */
lq_status lq_sim_set_fock(lq_sim* sim, int32_t chain, const int32_t* host_occ_up, const int32_t* host_occ_dn);
lq_status lq_sim_get_fock(lq_sim* sim, int32_t chain, int32_t* host_occ_up, int32_t* host_occ_dn);
/* Set the sweep counter of every chain (the Philox counter word). */
lq_status lq_sim_set_sweep_index(lq_sim* sim, uint32_t sweep);
/* n_sweeps sweeps of every chain, one persistent launch per plan class (one
 * CTA per chain, longest chains first).  A sweep samples the weight of Eq. 1:
 * an up pass of field updates (the fast-update ratio of SM Sec. VI, run as a
 * submatrix update), N_up then N_dn Fock-state swaps (ratio of Eq. 2 by the
 * QR update: removal Eqs. S9-S12, addition Eqs. S1-S8), and a down pass of
 * field updates with equal-time measurements at the block boundaries.
 * measure != 0 appends one record (LQ_NOBS sign-weighted means) per sweep.
 * Asynchronous on the stream. */
lq_status lq_sim_sweep(lq_sim* sim, int32_t n_sweeps, int32_t measure);
/* Autotune the batched launch (build-side tuning, no counterpart in the
 * paper).  A sweep runs one persistent launch per plan class: the chains with
 * at most 32 particles per spin, then the larger ones.  For each class this
 * times sweeps_per_candidate sweeps (without measurement) under each feasible
 * pair of (size of the shared-memory staging buffer, threads per CTA), and
 * keeps the fastest for later sweeps.  The staging size sets the
 * propagation's column chunks and the flip loop's chunk of sites; with the
 * threads per CTA (256, or 128 for the small class) it sets the CTAs, i.e.
 * the chains, resident per SM.  The timed sweeps are ordinary sweeps of the
 * chains of that class (they advance its chains; use them as warm-up), so a
 * class's chains advance by sweeps_per_candidate times the number of
 * candidates tried.  Choices are cached per (precision, class, N_sigma, N,
 * chain-count bucket) for the process; with sweeps_per_candidate = 0 only a
 * cached choice is applied.  host_buf2 (nullable) receives the staging bytes
 * chosen for the two classes (0 for an empty class).  Synchronous. */
lq_status lq_sim_autotune(lq_sim* sim, int32_t sweeps_per_candidate, int32_t* host_buf2);
/* The launch of each plan class as it stands (after lq_sim_create or
 * lq_sim_autotune): host_cfg8 = for the small then the large class, its
 * chains, staging bytes, threads per CTA and grid (zeros for an empty class). */
lq_status lq_sim_launch_config(const lq_sim* sim, int32_t* host_cfg8);
/* Pin the launch of plan class plan_class (0: at most 32 particles per spin,
 * 1: more) instead of the autotuner: staging bytes (at least the plan's
 * minimum) and threads per CTA (256; 128 allowed for class 0).  Errors:
 * LQ_EINVAL (bad class, empty class, bad sizes), LQ_EUNSUPPORTED (the
 * launch does not fit an SM or the simulation's workspace). */
lq_status lq_sim_set_launch_config(lq_sim* sim, int32_t plan_class, int32_t staging_bytes, int32_t threads);
/* One stateless batch call on host buffers: upload every chain's fields
 * (host_fields: chains concatenated, each L x N) and Fock state (host_occ:
 * each chain's n_up then n_dn sites), rebuild the QR chains, run n_sweeps
 * sweeps, and download the final fields, occupations (same layouts, either
 * output nullable) and the records of this call (host_records: each chain's
 * n_sweeps x LQ_NOBS, nullable; needs measure != 0).  Synchronous.  Fields
 * other than +-1 or repeated sites give LQ_EINVAL (checked on the device). */
lq_status lq_sim_run_host(lq_sim* sim, const int8_t* host_fields, const int32_t* host_occ, int32_t n_sweeps,
                          int32_t measure, int8_t* host_fields_out, int32_t* host_occ_out, double* host_records);
/* Wait for the stream; LQ_ENUMERIC if any chain flagged a numerical error. */
lq_status lq_sim_sync(lq_sim* sim);
/* log|W| and sign of chain c, W = prod_sigma det(P^T B(beta,0) P) of Eq. 1,
 * recomputed from freshly built QR chains (this also resets the tracked
 * weight). */
lq_status lq_sim_log_weight(lq_sim* sim, int32_t chain, double* log_abs, int32_t* sign);
/* log|W| and sign tracked through the accepted ratios since the last build. */
lq_status lq_sim_tracked_weight(lq_sim* sim, int32_t chain, double* log_abs, int32_t* sign);
/* Test hook: ratio W(s with s[slice][site] flipped) / W(s) (SM Sec. VI),
 * through the stabilized Green's function at that slice on freshly built
 * chains. */
lq_status lq_sim_field_ratio(lq_sim* sim, int32_t chain, int32_t slice, int32_t site, double* r);
/* Test hook: the Fock-state ratio of Eq. 2 for removing column k of spin
 * `spin` and adding site j (not occupied), by the Givens (Eq. S10) and
 * Gram-Schmidt (Eq. S7) QR update; parts (nullable, 6 doubles) = log|r|,
 * sign, log|r_remove|, sign, log|r_add|, sign. */
lq_status lq_sim_swap_ratio(lq_sim* sim, int32_t chain, int32_t spin, int32_t k, int32_t j, double* r,
                            double* parts);
/* Per-sweep records of chain c: *n_records rows of LQ_NOBS doubles into
 * host_out (capacity max_rows rows). */
lq_status lq_sim_records(lq_sim* sim, int32_t chain, int32_t max_rows, int32_t* n_records, double* host_out);
lq_status lq_sim_clear_records(lq_sim* sim);
/* counters of chain c: field attempts, field accepts, swap attempts, swap accepts */
lq_status lq_sim_stats(lq_sim* sim, int32_t chain, int64_t* host_counts4);
/* SM cycles chain c spent, summed over its sweeps, per phase: field flips,
 * slice propagation, QR restabilization, block-start Gram and inverse,
 * particle-hole swaps, measurement; then two parts of the swap cycles: the
 * removal (Givens rotations, M^-1, downdate, rotated Q panels) and the
 * addition (vector propagation and Gram-Schmidt); then four parts of the flip
 * cycles of chains with at most 32 particles per spin: row staging and
 * write-back, the products and blocks of each chunk's first window, the
 * leader warp's serial per-site chains, and the rest of the window loop (the
 * leader forming the next window's block and waiting for the other warps,
 * which meanwhile run the recurrences, the update of T and the next window's
 * products) (host array of 12). */
lq_status lq_sim_profile(lq_sim* sim, int32_t chain, int64_t* host_cycles12);
/* Test hook: panel j of the right (side 0) or left (side 1) chain of a spin,
 * as FP64 host arrays Q (N x N_sigma) and V (N_sigma x N_sigma, nullable). */
lq_status lq_sim_chain_panel(lq_sim* sim, int32_t chain, int32_t side, int32_t spin, int32_t j, double* host_Q,
                             double* host_V);
/* sizes of chain c: N, L, tau_w, n blocks, n_up, n_dn */
lq_status lq_sim_chain_info(const lq_sim* sim, int32_t chain, int32_t* info6);
/* device bytes held by the simulation */
lq_status lq_sim_device_bytes(const lq_sim* sim, size_t* bytes);
lq_status lq_sim_destroy(lq_sim* sim);

/* Numeric health check (build-side, no counterpart in the paper): rebuild
 * every chain's QR chains from its fields and Fock state, compare the fresh
 * log|W| and sign with the tracked ones (the running sum of accepted log|r|),
 * and keep the rebuilt chains, so the check also resynchronizes.  A chain
 * drifted if |fresh - tracked| / max(1, |fresh|) > tol or the signs differ.
 * host_max_rel / host_n_bad (nullable) receive the largest relative drift and
 * the number of drifted chains.  Errors: LQ_ENUMERIC when a chain drifted
 * (after resynchronizing it) or a device error flag is set; LQ_EINVAL for a
 * negative tol.  Synchronous; costs about one QR-chain build per chain. */
lq_status lq_sim_check_drift(lq_sim* sim, double tol, double* host_max_rel, int32_t* host_n_bad);

/* Sign-weighted means <sign O>/<sign> over chain c's per-sweep records and
 * their jackknife errors over n_bins bins (host arrays of LQ_NOBS; index 0
 * holds the mean sign and a zero error). */
lq_status lq_sim_measure(lq_sim* sim, int32_t chain, int32_t n_bins, double* host_mean, double* host_err);

/* ---- serving loop (continuous batching) -----------------------------------
 * A host thread owns one non-blocking CUDA stream on `device` and runs ticks:
 * admit queued requests first come first served while their device footprint
 * fits hbm_budget and fewer than max_active run; then ONE persistent launch
 * over every active request, each running its remaining sweeps within the
 * launch's time budget (see lq_server_set_tick_target); requests that arrive
 * while others run join the next launch; then retire requests that finished
 * their sweeps.  All requests share the server's precision.  Request arenas
 * come from a stream-ordered memory pool owned by the server, so admission
 * and retirement never synchronize the device. */
typedef struct lq_server lq_server;
typedef struct {
  const lq_lattice* lattice; /* copied at submit; the caller may destroy it */
  lq_params params;
  int32_t n_sweeps;          /* sweeps, each measured */
  uint32_t chain_id;         /* Philox chain word */
} lq_request;
typedef struct {
  int32_t status;            /* LQ_OK or the error that ended the request */
  int32_t n_records;
  double obs_mean[LQ_NOBS];  /* sign-weighted means, index 0 = mean sign */
  double obs_err[LQ_NOBS];   /* jackknife errors */
  double log_weight;         /* tracked log|W| at the end */
  int32_t sign;
  int64_t counts[4];         /* field attempts, accepts, swap attempts, accepts */
  double queue_ms;           /* submit -> admission */
  double total_ms;           /* submit -> retirement */
  double sweep_ms_mean;      /* mean device time of one of its sweeps */
  double wall_ms_per_sweep;  /* total_ms / sweeps: wall latency per sweep, queueing and batching included */
  int32_t active_at_admit;   /* requests already on the device when it was admitted */
  int32_t waited_for_memory; /* 1 if it reached the head of the queue and waited for memory to be freed */
} lq_result;
typedef struct {
  double p50_sweep_ms, p99_sweep_ms; /* per-sweep latency: one sample per sweep run, that sweep's own device time */
  double p50_tick_ms, p99_tick_ms;   /* duration of the batched launches */
  double updates_per_s;              /* field-update attempts per second of device busy time */
  double busy_s, wall_s;             /* device time of the batched launches; wall time since creation */
  double admit_s, retire_s;          /* host time spent admitting and retiring requests */
  int64_t submitted, admitted, completed, rejected, active, queued, ticks;
  size_t hbm_in_use;
  double p50_wall_sweep_ms, p99_wall_sweep_ms; /* over retired requests: (retirement - submission) / sweeps */
  int64_t sweeps;                              /* sweeps run */
} lq_server_info;
/* Percentiles come from fixed histograms (200 logarithmic bins per decade
 * from 1 us to 10^4 s, 1.2 % wide), so the statistics use constant memory. */
/* Device bytes a request of this lattice and these parameters holds while
 * it is admitted (fields, both QR chains, the stored block, scratch and
 * records): the amount the server charges against its budget.  Errors:
 * LQ_EINVAL for a null argument or parameters out of range. */
lq_status lq_request_footprint(const lq_lattice* lattice, const lq_params* params, size_t* bytes);
/* Errors: LQ_EINVAL for a bad budget, slot count, queue capacity or precision. */
lq_status lq_server_create(int32_t device, size_t hbm_budget, int32_t precision, int32_t max_active,
                           int32_t queue_capacity, lq_server** out);
/* Never blocks.  LQ_EBUSY when the queue is full; LQ_EINVAL when the request's
 * footprint exceeds the whole budget or its precision differs. */
lq_status lq_server_submit(lq_server* srv, const lq_request* request, uint64_t* id);
/* LQ_ENOTFOUND until the request is done; then fills *out once and forgets it. */
lq_status lq_server_poll(lq_server* srv, uint64_t id, lq_result* out);
lq_status lq_server_stats(lq_server* srv, lq_server_info* out);
/* Lower bound (ms) of the time budget of one batched launch (default 20).
 * Within a launch each request runs its remaining sweeps while they fit in
 * the budget, at least one; the budget is the longest expected single sweep
 * among the active requests and at least this target.  Larger targets mean
 * fewer launches and longer waits for newly admitted requests. */
lq_status lq_server_set_tick_target(lq_server* srv, double ms);
/* Finishes every admitted request, drops the queued ones, joins the thread. */
lq_status lq_server_destroy(lq_server* srv);

/* ---- constrained-path inner loop (SM Sec. VI) ------------------------------
 * For the Fock state eta given by its occupied sites (host arrays of n_up and
 * n_dn sites), walkers sample the Hubbard-Stratonovich fields slice by slice
 * against the trial Psi_l^T = P^T e^{-(beta - tau_l) H_0} (everything after
 * the fields of slice l, with the fields off).  At site i the overlap ratio
 * of field value s is r(s) = prod_sigma [1 + Delta_sigma(s) Phi_i (Psi^T
 * Phi)^{-1} Psi_i^T] (times e^{-lambda s} for U < 0); s is drawn with
 * probability proportional to (1/2) max(0, r(s)) and the walker's weight
 * takes the factor (1/2) sum_s max(0, r(s)); a walker at factor 0 has crossed
 * the trial's node and is dropped.  Without truncation the mean weight is
 * R(eta) = sum_s 2^{-LN} <eta|U(s)|eta> / <eta|e^{-beta H_0}|eta>, whose ratio
 * between Fock states corrects the free-fermion weight W_T(eta) that a U = 0
 * chain of lq_sim samples.  The paper fixes neither the field law nor the
 * population control: this is the plainest choice whose mean weight is
 * R(eta) when nothing is truncated.  params: the model (U, beta, dtau, n_up,
 * n_dn, kinetic, seed = Philox key); precision must be LQ_FP64
 * (LQ_EUNSUPPORTED otherwise); n_stab, swap_mode and left_swaps are not used.
 * Both calls allocate their device memory and synchronize.  Errors:
 * LQ_EINVAL (bad arguments or occupations), LQ_EUNSUPPORTED, LQ_ENOMEM,
 * LQ_ECUDA. */
/* n_walkers independent walkers; host_log_weights[k] = log of walker k's
 * final weight (-inf when dropped), host_dropped (nullable) the number
 * dropped.  Random numbers: Philox counter (k, sweep_word, 7<<24 | slice,
 * site). */
lq_status lq_cp_walk(const lq_lattice* lattice, const lq_params* params, const int32_t* host_occ_up,
                     const int32_t* host_occ_dn, int32_t n_walkers, uint32_t sweep_word, double* host_log_weights,
                     int32_t* host_dropped);
/* A branching population of n_walkers: after every comb_every slices (0: only
 * at the end) and after the last, the population's mean weight joins the
 * estimate and n_walkers new walkers (weight 1) are drawn from the old ones
 * by systematic (comb) resampling (Kitagawa 1996), probabilities
 * proportional to the weights.  *host_log_estimate = log of the product of
 * the mean weights (-inf if every walker was dropped), an unbiased estimate
 * of R(eta) when nothing is truncated.  Random numbers: Philox counters (slot,
 * run, 8<<24 | slice, site) for the fields and (run, 0xFFFFFFFD, 9<<24 | last
 * slice of the interval, 0) for the comb's uniform. */
lq_status lq_cp_population(const lq_lattice* lattice, const lq_params* params, const int32_t* host_occ_up,
                           const int32_t* host_occ_dn, int32_t n_walkers, int32_t comb_every, uint32_t run,
                           double* host_log_estimate);

/* ---- allocation-free single-chain sweep ----------------------------------
 * No counterpart in the paper: this entry point exists for callers that
 * cannot allocate device memory themselves, for example a plug-in that must
 * run inside a host framework which reserves all GPU memory up front, or code
 * that may not call cudaMalloc on a latency-critical path.  It runs n_sweeps
 * sweeps of ONE chain and allocates no device memory (and no host memory
 * unless it fails): the caller owns the inputs and outputs, and every scratch
 * buffer (QR chains, panels, lattice tables, the chain descriptor) lives in
 * one fixed array of LQ_NOALLOC_SCRATCH_BYTES in device memory, which each GPU
 * that loads the library holds until the process exits.
 *
 * dev_fields: device int8 L x N, +-1, updated in place.
 * dev_occ:    device int32, n_up then n_dn occupied sites (the columns of P),
 *             updated in place.
 * dev_records: device double n_sweeps x LQ_NOBS per-sweep records (nullable:
 *             no measurements).
 * sweep_index: the Philox sweep word of the first sweep (continue a chain by
 *             passing the previous index + n_sweeps).
 * host_log_weight / host_sign / host_counts4 (all nullable): if any is given,
 *             the call synchronizes the stream and returns the tracked
 *             log|W|, its sign, and the field/swap attempt and accept counts
 *             of this call.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls on a device share the scratch, which keeps the last call's
 * contents (every call rebuilds what it reads), so calls whose work overlaps
 * on the GPU race; serialize them on one stream.
 * Errors: LQ_EINVAL (bad arguments), LQ_EUNSUPPORTED (the chain needs more
 * scratch than LQ_NOALLOC_SCRATCH_BYTES, more than LQ_MAX_PARTICLES per spin,
 * or a shared-memory plan that does not fit one CTA per SM), LQ_ECUDA.  The
 * errors the kernels detect (LQ_EINVAL for fields other than +-1 or repeated
 * or out-of-range sites, LQ_ENUMERIC for a singular overlap, a CholeskyQR
 * breakdown or a non-finite ratio) can only be read back after the stream
 * has run, so they are reported only when a host output is requested; a call
 * with all three host outputs null returns LQ_OK for launched work. */
#define LQ_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
lq_status lq_sweep_noalloc(const lq_lattice* lattice, const lq_params* params, uint32_t chain_id,
                           uint32_t sweep_index, int8_t* dev_fields, int32_t* dev_occ, int32_t n_sweeps,
                           double* dev_records, void* cuda_stream, double* host_log_weight, int32_t* host_sign,
                           int64_t* host_counts4);

/* ---- device FP64 throughput (build-side, no counterpart in the paper) -----
 * The sweep's field-flip algebra is FP64 on the CUDA cores, so the roof it is
 * reported against is the device's FP64 FMA rate.  This measures it on the
 * current device: a kernel of independent FMA chains on every SM, grown until
 * one launch takes about `ms` milliseconds and timed with CUDA events, gives
 * *host_tflops (2 flops per FMA).  host_cycles9 (nullable, 9 doubles) receives
 * the sub-partition cycles of one FP64 FMA warp instruction with 1 and with 32
 * active lanes (eight independent chains) and of one FP32 FMA warp
 * instruction, then the latency in cycles of an instruction that depends on
 * the previous one: FP64 FMA, FP64 multiply, the FP64 reciprocal seed
 * rcp.approx.ftz.f64, an FP32 -> FP64 -> FP32 conversion pair, a 64-bit warp
 * shuffle, a dependent shared-memory load (one warp, clock64).
 * Allocates and frees a small device buffer; synchronous.
 * Errors: LQ_EINVAL (ms outside (0, 60000] or a null output), LQ_ECUDA. */
lq_status lq_device_fp64_rate(double ms, double* host_tflops, double* host_cycles9);
/* Gram probe (build-side, no counterpart in the paper): the sweep's dense
 * contractions are Grams W = A^T B of two N x m panels (the block Green's
 * function and the CholeskyQR2 Grams).  This times one Gram per CTA for
 * n_panels pairs of panels (the layout of the sweep: a CTA per chain) in one
 * of four forms: 0 the sweep's FP64 CUDA-core routine on FP64 panels, 1 the
 * FP64 tensor cores (DMMA, mma.sync m8n8k4) on FP64 panels, 2 the sweep's
 * CUDA-core routine on FP32 panels with FP64 accumulation (LQ_MIXED), 3 the
 * TF32 tensor cores with each FP32 operand split in two TF32 parts (three
 * products, FP32 accumulation) on FP32 panels.  *host_us = microseconds per
 * launch of n_panels Grams (CUDA events, mean of 5 after a warm-up);
 * *host_max_rel_err = the largest |W - W_ref| over the Gram's largest |entry|
 * against the FP64 CUDA-core Gram of the same values.  N >= 8, m a multiple
 * of 16 up to 128.  Allocates device memory; synchronous.  Errors:
 * LQ_EINVAL, LQ_ECUDA. */
lq_status lq_probe_gram(int32_t N, int32_t m, int32_t variant, int32_t n_panels, double* host_us,
                        double* host_max_rel_err);
/* Test hook (no counterpart in the paper): the field-flip loops form
 * c = Delta / (1 + Delta G_tt) with a hardware reciprocal seed and one
 * third-order Newton-Raphson step instead of the IEEE division sequence (the
 * four-warp path as the quotient d / r, the paired path as the reciprocal
 * 1 / (1/Delta + G_tt), which is this quotient at d = 1 bit for bit).  This
 * evaluates that quotient and the IEEE quotient d[k] / r[k] on the device for
 * n host operand pairs (host arrays of n; outputs host arrays of n).
 * Allocates device memory; synchronous.  Errors: LQ_EINVAL, LQ_ECUDA. */
lq_status lq_test_quotient(int32_t n, const double* host_d, const double* host_r, double* host_q,
                           double* host_q_ieee);

const char* lq_last_error(void);
const char* lq_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LECQMC_H */
