/*
 * hf_oracle.h -- plain, slow, FP64 CPU oracle for the Hirsch-Fye QMC impurity
 * solver used inside real-space DMFT (Bluemer & Gorelik, "Quantum Monte Carlo
 * simulations of antiferromagnetism in ultracold fermions on optical lattices
 * within real-space dynamical mean-field theory", arXiv:1006.2716).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this code; only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark do.  It shares no code,
 * header, table or constant generator with the CUDA implementation.
 *
 * Conventions (positive Green function, g_{ll'} = <T c(tau_l) c^dagger(tau_l')>,
 * tau_l = l * dtau, diagonal taken at tau -> 0+ so that g_ll = 1 - n):
 *   - Trotter step dtau = beta / L, Ising fields s_l = +-1, cosh(lambda) = exp(dtau U / 2)
 *     ("Model and Methods": Hirsch-Fye solver with a fixed dtau; the decoupling of
 *     U (n_up n_dn - (n_up + n_dn)/2) by one Ising field per slice).
 *   - V^sigma_l = lambda * sigma * s_l with sigma = +1 (up), -1 (down).
 *   - Dyson relation G = [1 + (1 - g0)(e^V - 1)]^{-1} g0.
 *   - single-flip ratio R_sigma = 1 + (1 - G_ll)(e^{-2 lambda sigma s_l} - 1),
 *     Metropolis acceptance u < R_up R_dn, Sherman-Morrison rank-1 update.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter
 *     (sweep, l, chain, site), key (seed_lo, seed_hi); sweep 0xFFFFFFFF draws the
 *     initial fields.
 * All matrices are L x L, row-major, element (i, j) at i * L + j.
 */
#ifndef HF_ORACLE_H
#define HF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32 with 10 rounds, as published by Salmon et al. (SC'11). */
void hfo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* 53-bit uniform in [0, 1) for proposal (sweep, l) of (site, chain):
 * ((x0 << 32 | x1) >> 11) * 2^-53 of the Philox block. */
double hfo_uniform(uint64_t seed, uint32_t site, uint32_t chain, uint32_t sweep, uint32_t l);

/* Initial Ising fields: s_l = +1 if the top bit of x0 (counter (0xFFFFFFFF, l, chain, site))
 * is clear, else -1. */
void hfo_init_fields(uint64_t seed, uint32_t site, uint32_t chain, int L, int8_t* s);

/* dtau = beta / L and lambda = acosh(exp(dtau U / 2)). */
void hfo_constants(double beta, double U, int L, double* dtau, double* lambda);

/* Antiperiodic Toeplitz bath matrix from g0(tau_m), m = 0..L-1 (tau_0 = 0+):
 * g0[l][l'] = gt[l - l'] for l >= l', -gt[l - l' + L] for l < l'. */
void hfo_build_g0(int L, const double* gt, double* g0);

/* Dyson refresh: G = A^{-1} g0 with A = 1 + (1 - g0) diag(exp(lambda sigma s) - 1),
 * by Gaussian elimination with partial pivoting.  Writes det(A) to *det if det != 0.
 * Returns 0, or -1 if A is singular. */
int hfo_dyson(int L, const double* g0, const int8_t* s, int sigma, double lambda,
              double* G, double* det);

/* Single-flip ratio of slice l: a[sp] = exp(-2 lambda sigma s_l) - 1 and
 * R[sp] = 1 + (1 - G_sigma[l][l]) a[sp] for sp = 0 (up, sigma = +1), 1 (down, sigma = -1).
 * Returns the Metropolis weight ratio R_up * R_dn. */
double hfo_ratio(int L, double lambda, const int8_t* s, int l, const double* Gup,
                 const double* Gdn, double* a, double* R);

/* One sweep l = 0..L-1 over one chain, rank-1 Sherman-Morrison updates in place.
 * Returns the number of accepted flips. */
int hfo_sweep(int L, double lambda, uint64_t seed, uint32_t site, uint32_t chain,
              uint32_t sweep, int8_t* s, double* Gup, double* Gdn);

/* Near-tie watch: from now on count the proposals of hfo_sweep whose uniform u lies within
 * rel * |R_up R_dn| of R_up R_dn (rel = 0 switches it off); hfo_tie_count returns the count.
 * Process-wide state, not thread safe; it changes no result. */
void hfo_tie_watch(double rel);
long hfo_tie_count(void);

/* Accumulate one measurement of G into acc: layout acc[0..L-1] = G_up(tau_m),
 * acc[L..2L-1] = G_dn(tau_m), acc[2L] = n_up, acc[2L+1] = n_dn, acc[2L+2] = double
 * occupancy.  G_sigma(tau_m) = (1/L) sum_l sgn G[(l+m) mod L][l], sgn = -1 on wrap. */
void hfo_measure(int L, const double* Gup, const double* Gdn, double* acc);

/* Run one chain: for k in [0, n_warmup + n_measure): sweep number *nsw, then
 * (*nsw)++, a Dyson refresh of both spins whenever (*nsw + phase) % refresh_every == 0
 * (phase = 0, or (site + chain) % refresh_every when refresh_stagger is 1: the refresh
 * interval is the same for every chain, its offset differs), and, for k >= n_warmup, a
 * measurement added to bin (k - n_warmup) / bin_size of bins[nbins][2L+3] (bins must be
 * zeroed by the caller when a fresh run starts).
 * Gup/Gdn must hold the Green functions that belong to s on entry.
 * Returns accepted flips, or -1 on a singular refresh. */
long hfo_run_chain(int L, double lambda, const double* g0up, const double* g0dn,
                   uint64_t seed, uint32_t site, uint32_t chain, uint32_t* nsw,
                   int n_warmup, int n_measure, int refresh_every, int refresh_stagger,
                   int bin_size, int8_t* s, double* Gup, double* Gdn, double* bins);

/* Exact discretised averages by enumeration of all 2^L field configurations
 * (L <= 20): weights w(s) = det A_up(s) det A_dn(s), observables as hfo_measure.
 * out[2L+3] = sum_s w(s) O(s) / sum_s w(s).  Returns 0 or -1. */
int hfo_brute_force(int L, double lambda, const double* g0up, const double* g0dn, double* out);

#ifdef __cplusplus
}
#endif
#endif
