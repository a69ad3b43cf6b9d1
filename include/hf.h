/*
 * hf.h -- C ABI of the GB300 (sm_103a) Hirsch-Fye QMC / real-space DMFT library.
 *
 * Method: N. Bluemer and E. V. Gorelik, "Quantum Monte Carlo simulations of
 * antiferromagnetism in ultracold fermions on optical lattices within real-space
 * dynamical mean-field theory" (arXiv:1006.2716).
 *   - eq. 1: trapped Hubbard model, hopping t, on-site U, trap V_i = V0 r_i^2, chemical
 *     potential mu.
 *   - eq. 2: lattice Green function [G(i w_n)]^{-1}_ij = t_ij + [i w_n + mu - V_i -
 *     Sigma_i(i w_n)] delta_ij with a site-diagonal self-energy, one frequency at a time.
 *   - "Model and Methods": one Anderson impurity problem per inequivalent site, solved by
 *     Hirsch-Fye QMC at a fixed Trotter step dtau; importance sampling over many Markov
 *     chains per impurity.
 *
 * Conventions shared by every entry point:
 *   - Green functions are in the positive convention g(tau) = <T c(tau) c^dagger(0)>, so
 *     g(0+) = 1 - n.  Imaginary times tau_m = m dtau, m = 0..L-1, L = round(beta / dtau).
 *   - Spin index 0 = up (sigma = +1), 1 = down (sigma = -1).
 *   - Every call returns an hf_status; nothing is thrown or exits across the ABI.  The text
 *     of the last failure of a context is returned by hf_last_error.
 *   - Device memory is never allocated by the library: hf_init takes a caller-owned device
 *     workspace of hf_workspace_size bytes (256-byte aligned) and keeps its state in it;
 *     the caller keeps that buffer alive until hf_free.  Host buffers passed to calls are
 *     owned by the caller and only read or written during the call.
 *   - All device work is queued on params.cuda_stream (a cudaStream_t; NULL = the legacy
 *     default stream).  Calls that return host data synchronise that stream.
 */
#ifndef HF_H
#define HF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HF_OK = 0,
    HF_EINVAL = -1,    /* bad argument or parameter combination                        */
    HF_ENOMEM = -2,    /* workspace too small                                          */
    HF_ECUDA = -3,     /* a CUDA runtime call failed                                   */
    HF_ETIMEOUT = -4,  /* a bounded device wait ran out                                */
    HF_ENUMERIC = -5,  /* singular Dyson matrix or non-finite value detected on device */
    HF_EBUSY = -6,     /* no free slot / resource                                      */
    HF_ENOTREADY = -7  /* requested result is not available yet                        */
} hf_status;

typedef struct hf_ctx hf_ctx;

/* Parameters of one trapped-lattice RDMFT problem (eq. 1 plus the QMC settings). */
typedef struct hf_params {
    int Lx, Ly;          /* geometry 0: Lx x Ly square; geometry 1: disc of radius Lx       */
    int Lz;              /* geometries 2, 3: layers (ignored in two dimensions)              */
    int geometry;        /* 0 square (centre ((Lx-1)/2, (Ly-1)/2)), 1 site-centred disc,     */
                         /* 2 Lx x Ly x Lz box with a spherical trap about its centre,       */
                         /* 3 slab of Lz layers with a cylindrical trap V0 (dx^2 + dy^2),    */
                         /* periodic across the layers ("Efficient simulations for three     */
                         /* dimensions").  Sites (x, y, z) are numbered (z Ly + y) Lx + x.   */
    int periodic;        /* 1: periodic boundaries (square; box: all axes; slab: x and y),   */
                         /* measured trap from the box centre; 0: open.  A periodic axis of  */
                         /* the box or slab needs an even length >= 4                       */
    double t, U, V0, mu; /* eq. 1: hopping, interaction, trap strength, chemical potential  */
    double beta, dtau;   /* inverse temperature, Trotter step; L = round(beta / dtau)       */
    int n_matsubara;     /* Matsubara frequencies kept explicitly (paper: 500)              */
    int chains_per_site; /* independent Markov chains per inequivalent site                 */
    int precision;       /* 0: FP64 sweeps; 1: FP32 sweeps + FP64 refresh; 2: FP32-pair     */
                         /* ("double-float", 48-bit significand) sweeps + FP64 refresh      */
    int refresh_every;   /* Dyson refresh after every refresh_every-th sweep of a chain     */
    int refresh_stagger; /* 0: a chain refreshes when its sweep counter n is a multiple of   */
                         /* refresh_every; 1: when n + site + chain is (site, chain = the    */
                         /* Philox counter words), so the FP64 refreshes of chains that run  */
                         /* side by side fall on different sweeps; needs precision 0 or 2    */
                         /* unless refresh_every is 1                                       */
    int check_drift;     /* 1: at every refresh within a sweep launch, measure how far the    */
                         /* updated G has drifted from the Dyson solution that replaces it   */
                         /* (hf_get_drift); 0: off.  The chains' arithmetic is unchanged     */
    int refresh_gj;      /* precision 1 at L = 128: 0 (default) refreshes after each sweep by */
                         /* two Newton steps on the tensor cores (products formed exactly     */
                         /* from bf16 digits), falling back to Gauss-Jordan for a chain whose */
                         /* residual does not converge; 1 always uses FP64 Gauss-Jordan       */
    int lattice_form;    /* lattice step (eq. 2): 0 (default) picks by band half-width b: below */
                         /* 128 the band L D L^T and selected inversion in a shared-memory    */
                         /* window, from 128 on (up to 840) the blocked band L D L^T in global */
                         /* memory with G_ii from forward solves L^{-1} e_i at one site per    */
                         /* orbit and spin (for 128 <= b <= 520 its products run as exact    */
                         /* bf16 digit products on the tensor cores, each entry rounded once */
                         /* to FP64); 1 always takes the blocked band form; 2 always the      */
                         /* window form (b <= 165, HF_EINVAL above)                            */
    int delay_k;         /* delayed-update depth: 0/1 rank-1 Sherman-Morrison; 4, 8, 16, 32  */
                         /* (precision 2, one warp per chain): accepted flips gathered as    */
                         /* rank-k corrections                                              */
    int team_warps;      /* FP64-class sweeps: warps per Markov chain, 1, 2 or 4 (0: default */
                         /* 1 for L <= 32, 4 above); picked per L by the autotuner          */
    int bin_size;        /* measured sweeps per bin                                         */
    int max_bins;        /* bins kept per chain between clears                              */
    int n_warmup, n_measure;  /* sweeps per hf_rdmft_step                                  */
    uint64_t seed;       /* Philox key                                                      */
    double h_seed;       /* staggered seed field of iteration 0                             */
    double mix;          /* linear self-energy mixing                                       */
    void* cuda_stream;   /* cudaStream_t used for every device operation                    */
} hf_params;

/* Bytes of device workspace hf_init needs for *p (*bytes set on HF_OK). */
hf_status hf_workspace_size(const hf_params* p, size_t* bytes);

/* Host only, no device work: the lattice *p describes (after the same validation as hf_init).
 * Writes the number of sites, of inequivalent sites, the band half-width of H0 that the lattice
 * step factors, and the matrices it inverts per Matsubara frequency (2; or 1 when a symmetry of
 * the lattice exchanges the two sublattices, so that the spin-down G_ii are spin-up ones at
 * permuted sites); rep [n_sites], rep_of [N] and flip [N] (as in hf_get_orbits) when not NULL --
 * call once with them NULL to learn the sizes.  HF_EINVAL for invalid parameters or a band wider
 * than the lattice step supports. */
hf_status hf_lattice_info(const hf_params* p, int* N, int* n_sites, int* band, int* spins, int* rep,
                          int* rep_of, int* flip);

/* Validate *p, build the lattice (eq. 1) and its point-group orbits (C4v in two dimensions,
 * the cubic group for the box, the planar group with the layer translations for the slab), lay
 * the state out in the caller's device workspace d_ws (ws_bytes >= hf_workspace_size), draw the
 * initial Ising fields of every chain and seed Sigma_{i,sigma}(i w_n) = U/2 - sigma h_seed
 * eps_i.  *out receives a host handle released by hf_free.  HF_EINVAL for invalid parameters,
 * including a lattice whose band half-width in the lattice step's band order (periodic axes
 * folded) exceeds 840, the widest band the blocked band form keeps buffers for; HF_ENOMEM for
 * a workspace smaller than hf_workspace_size. */
hf_status hf_init(const hf_params* p, void* d_ws, size_t ws_bytes, hf_ctx** out);

/* Number of inequivalent sites, chains, L, lattice sites N (any pointer may be NULL). */
hf_status hf_get_sizes(const hf_ctx* ctx, int* n_sites, int* n_chains, int* L, int* N);

/* Orbit tables: rep[n_sites] = lattice index of each inequivalent site; rep_of[N] =
 * inequivalent index of every lattice site; flip[N] = 1 if that site sits on the other
 * sublattice than its representative (its spins are exchanged).  Host buffers. */
hf_status hf_get_orbits(const hf_ctx* ctx, int* rep, int* rep_of, int* flip);

/* Set the Hartree-shifted bath g~0_sigma(tau_m), m = 0..L-1 (tau_0 = 0+), of one
 * inequivalent site and spin from a host array of L doubles.  The next hf_sweep with
 * refresh_first = 1 rebuilds every chain of that site from it (Dyson relation); the inverse
 * bath matrices the refreshes use are recomputed before that sweep.  Every site's bath must
 * be set before sweeping (a zero bath matrix has no inverse: HF_ENUMERIC). */
hf_status hf_set_g0(hf_ctx* ctx, int site, int spin, const double* g0_tau);

/* Run n_warmup unmeasured then n_measure measured sweeps of every chain (asynchronous on
 * the context stream).  refresh_first = 1 first recomputes G = [1 + (1 - g0)(e^V - 1)]^{-1} g0
 * from the current bath and fields (in FP64, as G = [g0^{-1} e^V - (e^V - 1)]^{-1}).  Per chain: sweep number w uses Philox counter
 * (w, l, chain, site); after the sweep the chain's counter advances and a Dyson refresh runs
 * when it is a multiple of refresh_every; measured sweeps then add to the current bin. */
hf_status hf_sweep(hf_ctx* ctx, int n_warmup, int n_measure, int refresh_first);

/* Zero all measurement bins and counters (the next measured sweep starts bin 0), the drift
 * monitor and the refresh counters of hf_get_refresh_stats. */
hf_status hf_clear_measurements(hf_ctx* ctx);

/* Reduce the completed bins of every chain of one inequivalent site (synchronises):
 * gtau[2][L] = G_sigma(tau_m), n[2] = densities, d = double occupancy, m = n_up - n_dn, each
 * averaged over chains x bins; errs[2L + 4] = standard errors in the same order
 * (gtau_up, gtau_dn, n_up, n_dn, d, m).  Any output pointer may be NULL. */
hf_status hf_measure(hf_ctx* ctx, int site, double* gtau, double* n, double* d, double* m,
                     double* errs);

/* One full RDMFT iteration on the device: lattice step (eq. 2) for every frequency and
 * spin, Weiss fields and their tau transform, warm-started QMC (n_warmup + n_measure sweeps),
 * chain/bin reduction, tau -> i w transform, Sigma = 1/G0 - 1/G_imp and mixing.  Writes the
 * wall time of the iteration to *iter_seconds (may be NULL).  Synchronises. */
hf_status hf_rdmft_step(hf_ctx* ctx, double* iter_seconds);

/* The first two phases of hf_rdmft_step alone: lattice step (eq. 2) from the current
 * self-energy, Weiss fields and the tau-grid baths g~0(tau_m) of every inequivalent site
 * (readable with hf_get_g0 / hf_get_gloc); no sweeps.  Synchronises. */
hf_status hf_compute_baths(hf_ctx* ctx);

/* Self-energy of the inequivalent sites, [n_sites][2][n_matsubara] complex as interleaved
 * (re, im) doubles; get copies it to the host, set replaces it from the host. */
hf_status hf_get_sigma(hf_ctx* ctx, double* sigma);
hf_status hf_set_sigma(hf_ctx* ctx, const double* sigma);

/* Observables of the last hf_rdmft_step or hf_measure: per inequivalent site
 * [n_sites][2L + 4] means and errors in the hf_measure order.  Synchronises. */
hf_status hf_get_observables(hf_ctx* ctx, double* mean, double* err);

/* Lattice-step output of the last hf_rdmft_step: G_ii(i w_n) of the inequivalent sites,
 * [n_sites][2][n_matsubara] complex (re, im interleaved).  Synchronises. */
hf_status hf_get_gloc(hf_ctx* ctx, double* gloc);

/* Bath g~0(tau_m) currently set, [n_sites][2][L].  Synchronises. */
hf_status hf_get_g0(hf_ctx* ctx, double* g0_tau);

/* Frequency-domain quantities of the last hf_rdmft_step, each [n_sites][2][n_matsubara]
 * complex (re, im interleaved), any pointer NULL to skip: the shifted Weiss field
 * G~0(i w_n) = 1/(1/G0 - U/2) the bath was built from, 1/G0 = 1/G_ii + Sigma, the impurity
 * G(i w_n) transformed from the measured G(tau) ("Model and Methods": G_imp = G~0 +
 * FT[-spline(g_imp - g~0)]), and the new self-energy 1/G0 - 1/G_imp before mixing.
 * Synchronises. */
hf_status hf_get_impurity_iw(hf_ctx* ctx, double* gw0, double* weiss_inv, double* gimp,
                             double* sigma_new);

/* Checkpoint / resume: fields [n_chains][L] int8 (+-1), per-chain sweep counters
 * [n_chains].  Setting fields invalidates G until the next refresh (hf_sweep with
 * refresh_first = 1).  Synchronises. */
hf_status hf_get_fields(hf_ctx* ctx, signed char* fields, uint32_t* sweep_counters);
hf_status hf_set_fields(hf_ctx* ctx, const signed char* fields, const uint32_t* sweep_counters);

/* Green-function matrices of one chain, [2][L][L] row-major doubles (converted from the
 * single-precision or FP32-pair state when precision = 1 or 2), and accepted-flip counters
 * [n_chains]. */
hf_status hf_get_green(hf_ctx* ctx, int chain, double* G);
hf_status hf_get_accepts(hf_ctx* ctx, unsigned long long* accepts);

/* Numerical-drift monitor (hf_params.check_drift = 1): the largest max_ij |G_SM - G_Dyson| over
 * every chain, spin and refresh inside the sweep launches since the last
 * hf_clear_measurements, where G_SM is the state the Sherman-Morrison updates reached and G_Dyson
 * the FP64 Dyson solution that replaces it (both as stored: FP64, FP32 pairs or FP32), and the
 * number of chain refreshes checked.  The refresh at the start of a launch is not checked (the
 * bath may have changed).  Either pointer may be NULL.  Synchronises. */
hf_status hf_get_drift(hf_ctx* ctx, double* max_drift, unsigned long long* refreshes);

/* The lattice step of this context (eq. 2; host only): *form 0 = band L D L^T with selected
 * inversion in a shared-memory window (every diagonal element), 1 = blocked band L D L^T in
 * global memory with forward solves L^{-1} e_k at the listed positions (see lattice_form);
 * *launches = kernel launches per lattice step; *cfma = complex multiply-adds that the form's
 * algorithm performs per (w_n, sigma) matrix (factorisation plus selected inversion, or plus
 * the forward solves), averaged over the spin matrices; *tc_flops = bf16 flops per matrix of
 * the exact digit products with which the blocked form runs its panels, trailing updates and
 * forward solves on the tensor cores (band half-widths 128 .. 520; 0 otherwise), averaged over
 * the spin matrices.  Any pointer may be NULL. */
hf_status hf_get_lattice_plan(const hf_ctx* ctx, int* form, int* launches, double* cfma,
                              double* tc_flops);

/* Refreshes of the mixed-precision form at L = 128 since the last hf_clear_measurements: chains
 * refreshed by the Newton steps on the tensor cores; chains those steps handed to the FP64
 * Gauss-Jordan refresh (a residual that did not converge, or a G too badly conditioned for the
 * residual's fixed-point accuracy); and the 128 x 128 x 128 digit products the steps ran on the
 * tensor cores (2 * 128^3 bf16 flops each).  Any pointer may be NULL.  Synchronises. */
hf_status hf_get_refresh_stats(hf_ctx* ctx, unsigned long long* tensor_refreshes,
                               unsigned long long* fallbacks, unsigned long long* digit_products);

/* Waits for the context stream and reports any failure the device recorded (numerical, or a
 * self-check of a checking build).  */
hf_status hf_sync(hf_ctx* ctx);

/* Device time in milliseconds, from CUDA events recorded on the context stream, of the phases
 * of the last hf_rdmft_step: ms[0] lattice step, ms[1] Weiss fields + i w -> tau, ms[2] QMC
 * sweeps, ms[3] chain/bin reduction, ms[4] tau -> i w + self-energy update; ms[5] the QMC
 * sweeps of the last hf_sweep.  A phase that has not run yet reads -1.  Synchronises. */
hf_status hf_get_timings(hf_ctx* ctx, double* ms);

/* ---- Batches: uneven-L problems in one fused launch, graph-captured iterations -------------
 * A batch groups 1..16 contexts that share one stream, one sweep form (precision 0 or 2, not 1)
 * and the same n_warmup / n_measure -- e.g. one RDMFT run per temperature of a scan, each with its
 * own L.  The impurity sweeps of all of them run as a single launch of the fused sweep kernel
 * (problems ordered by L, largest first, so the longest chains start first); every other phase
 * of an iteration stays per context.  The caller keeps the contexts alive until hf_batch_free. */
typedef struct hf_batch hf_batch;

/* use_graph = 1: from the second hf_batch_rdmft_step on, the whole iteration (lattice steps,
 * transforms, fused sweeps, reductions, self-energy updates) is replayed from one CUDA graph
 * captured on the first replayed call; the contexts' stream must then be a created stream (not
 * the legacy default stream), else HF_EINVAL. */
hf_status hf_batch_create(hf_ctx* const* ctxs, int n, int use_graph, hf_batch** out);

/* Fused sweeps of every context (asynchronous; same semantics per context as hf_sweep). */
hf_status hf_batch_sweep(hf_batch* b, int n_warmup, int n_measure, int refresh_first);

/* One RDMFT iteration of every context of the batch (as hf_rdmft_step for each); writes the
 * device time of the whole batched iteration in milliseconds to *gpu_ms (may be NULL).
 * Synchronises. */
hf_status hf_batch_rdmft_step(hf_batch* b, double* gpu_ms);

/* Device time (ms) of the last hf_batch_sweep or hf_batch_rdmft_step.  Synchronises. */
hf_status hf_batch_elapsed(hf_batch* b, double* gpu_ms);

void hf_batch_free(hf_batch* b);
const char* hf_batch_last_error(const hf_batch* b);

/* ---- Serving: continuously batched impurity solves ----------------------------------------
 * A service object accepts Hirsch-Fye impurity solves (one inequivalent site of one RDMFT run,
 * its bath g~0(tau) and L) from any host thread.  A scheduler thread inside the library admits
 * queued requests in arrival order whenever the device memory they need (chains x (2 L^2 FP64
 * entries + fields + bins), first-fit in the caller's device pool) and one of its streams are
 * free; up to requests_per_launch admitted requests share one launch of the fused sweep kernel,
 * and launches on different streams overlap on the GPU, so requests that arrive while others run
 * start without waiting for them.  The Ising fields and sweep counters of each (run, site) key
 * stay on the device between its requests (warm start; a key's next request waits for its
 * previous one); a request whose L differs from the L of the key's kept fields starts cold, and
 * its fields then replace the kept ones; with more keys than max_keys the least recently used
 * idle key is dropped and its next request starts cold.  Chains are keyed by (seed, site, chain) and computed exactly as
 * in a context of their own, so a result does not depend on which requests shared its launch.
 * No device code waits or polls: all waiting is on the host, with timeouts. */
typedef struct hf_srv hf_srv;

typedef struct hf_srv_params {
    int chains_per_request;   /* Markov chains per impurity solve                           */
    int n_warmup, n_measure;  /* sweeps per solve (n_measure a multiple of bin_size)        */
    int refresh_every;        /* FP64 Dyson refresh cadence (sweeps)                        */
    int refresh_stagger;      /* 1: per-chain refresh phases, as hf_params.refresh_stagger  */
    int bin_size;             /* measured sweeps per bin                                    */
    int precision;            /* 0 FP64 sweeps, 2 FP32-pair sweeps (both FP64 refresh)      */
    int team_warps;           /* warps per chain (0: default)                               */
    int max_L;                /* largest L admitted (<= 64)                                 */
    int max_inflight;         /* requests on the device at once                             */
    int max_keys;             /* warm-start records kept on the device                      */
    int n_streams;            /* concurrent launches                                        */
    int requests_per_launch;  /* requests fused into one launch (<= 16; 0: 16)              */
} hf_srv_params;

typedef struct hf_request {
    int run, site;            /* warm-start key; site is also the Philox site word          */
    int L;                    /* time slices, supported L <= max_L                          */
    double beta, U;           /* dtau = beta / L, cosh(lambda) = exp(dtau U / 2)            */
    uint64_t seed;            /* Philox key of this run's chains                            */
    double g0_tau[2][64];     /* Hartree-shifted bath, g0_tau[spin][m], m < L               */
} hf_request;

typedef struct hf_result {
    uint64_t ticket;
    int status;               /* HF_OK or the failure of this solve                         */
    int L;
    int warm;                 /* 1 if the chains continued from kept fields                 */
    uint32_t sweeps_done;     /* sweep counter of chain 0 after this solve                  */
    double gtau[2][64];       /* G_sigma(tau_m), mean over chains x bins                    */
    double n[2], d, m;        /* densities, double occupancy, n_up - n_dn                   */
    double err[2 * 64 + 4];   /* standard errors: gtau_up[L], gtau_dn[L], n_up, n_dn, d, m  */
    double latency_s;         /* submit -> result available                                 */
} hf_result;

typedef struct hf_srv_stats_t {
    int queued, inflight, peak_inflight, warm_keys;
    uint64_t completed;
    size_t bytes_in_use, peak_bytes, arena_bytes;
} hf_srv_stats_t;

/* Device pool bytes for the warm-start store plus max_inflight requests at max_L. */
hf_status hf_srv_workspace_size(const hf_srv_params* p, size_t* bytes);
/* Starts the service on the current device with the caller's 256-byte-aligned device pool
 * (kept alive by the caller until hf_srv_free).  Creates its own streams and pinned host
 * staging. */
hf_status hf_srv_create(const hf_srv_params* p, void* d_pool, size_t pool_bytes, hf_srv** out);
/* Queues a solve (copied); returns at once with a ticket. */
hf_status hf_srv_submit(hf_srv* s, const hf_request* r, uint64_t* ticket);
/* HF_OK and *out filled once the ticket's result exists (then forgotten), HF_ENOTREADY before. */
hf_status hf_srv_poll(hf_srv* s, uint64_t ticket, hf_result* out);
/* As hf_srv_poll, waiting up to timeout_s seconds (HF_ETIMEOUT after). */
hf_status hf_srv_wait(hf_srv* s, uint64_t ticket, double timeout_s, hf_result* out);
hf_status hf_srv_stats(hf_srv* s, hf_srv_stats_t* out);
/* Drops queued requests, lets admitted launches finish, stops the scheduler thread. */
void hf_srv_free(hf_srv* s);
const char* hf_srv_last_error(const hf_srv* s);

/* Allocation-free lattice step.  The paper has no counterpart: this exists for callers that
 * cannot allocate device memory at call time -- code running where a cudaMalloc would
 * synchronise the device or is forbidden (inside a latency-critical loop, or under a host
 * framework whose allocator owns all device memory and only hands out the caller's own input and
 * output buffers).  It computes exactly what the lattice phase of hf_rdmft_step computes,
 * G_ii(i w_n) = [(i w_n + mu) 1 - H0 - Sigma(i w_n)]^{-1}_ii of the inequivalent sites for every
 * frequency and spin, but keeps its band buffers in a fixed 16 MiB device array inside the
 * library instead of the workspace.
 *   d_sigma: device, [n_sites][2][n_matsubara] complex (re, im interleaved), read only.
 *   d_gloc:  device, same layout, written.
 * The lattice tables come from ctx; work is queued on the context stream and the call
 * synchronises it.  It allocates nothing (no cudaMalloc/cudaFree, no library allocator).
 * Limits and sharing: a lattice whose band (N * (b + 1) * 16 bytes, b = band half-width) exceeds
 * 16 MiB is rejected with HF_EINVAL; frequencies are processed in chunks that fit.  Every GPU
 * that loads the library holds the 16 MiB until the process exits.  All calls share the one
 * array, which keeps the last call's contents (every element is rewritten before it is read, so
 * nothing needs clearing); calls that overlap on the GPU -- e.g. from two streams -- race.  The
 * first call on a device looks the array's device address up (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture. */
hf_status hf_lattice_step_noalloc(hf_ctx* ctx, const double* d_sigma, double* d_gloc);

/* Raw blocks of the device random-number generator every sweep draws from: Philox4x32-10
 * (Salmon, Moraes, Dror and Shaw, SC'11), the counter-based generator the sweeps key by (sweep,
 * slice, chain, site).  For k < n, writes the four 32-bit words of the block at counter
 * d_ctr[4k .. 4k+3] under key (key_lo, key_hi) to d_out[4k .. 4k+3].  d_ctr and d_out are device
 * buffers of 4n uint32 each (the caller's, 16-byte aligned); the work is queued on cuda_stream (a cudaStream_t,
 * NULL = the legacy default stream) and the call does not synchronise.  HF_EINVAL for n < 0, or
 * for a null or unaligned buffer with n > 0; HF_ECUDA if the launch fails. */
hf_status hf_philox_blocks(uint32_t key_lo, uint32_t key_hi, const uint32_t* d_ctr, int n,
                           uint32_t* d_out, void* cuda_stream);

/* FP64-accurate products of 128 x 128 matrices on the tensor cores, the building block of the
 * L = 128 refresh: C_b = A_b B_b for b < n, row-major FP64 matrices of 128 x 128 doubles at
 * d_A + 16384 b, d_B + 16384 b, d_C + 16384 b (device buffers, the caller's, 16-byte aligned).
 * Every row of A and column of B is scaled by a power of two and cut into `digits` (1, 3, 5, 7 or
 * 8) balanced base-256 digits, exact in bf16; the digit products of the levels s + t <= digits + 1
 * are summed exactly in FP32 tensor-core accumulators and combined in 64-bit integers.  The error
 * of C_ij is below about 2^(9 - 8 digits) of 2^(TA_i + TB_j), the operands' row and column scales
 * (|A_ik| <= 2^(TA_i - 1), |B_kj| <= 2^(TB_j - 1)); 8 digits hold the operands' 62-bit fixed-point
 * forms exactly.  d_status (device int, may be NULL)
 * receives HF_ETIMEOUT if a bounded wait for the tensor cores ran out.  Asynchronous on
 * cuda_stream.  HF_EINVAL for n < 0, an unsupported digit count or a null or unaligned buffer. */
hf_status hf_tc_dgemm128(const double* d_A, const double* d_B, double* d_C, int n, int digits,
                         int* d_status, void* cuda_stream);

/* Release the host handle (the device workspace stays the caller's). */
void hf_free(hf_ctx* ctx);

/* Text of the last error of ctx (or of the last hf_init failure if ctx is NULL). */
const char* hf_last_error(const hf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HF_H */
