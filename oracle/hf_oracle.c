/*
 * hf_oracle.c -- plain FP64 CPU oracle of the Hirsch-Fye QMC impurity solver
 * (arXiv:1006.2716, "Model and Methods": each inequivalent site of the trapped
 * lattice is an Anderson impurity solved by Hirsch-Fye QMC at fixed dtau).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
 * CPU-baseline leg; never by the product path.  Deliberately unoptimised: every
 * step is written in the order the algorithm states it, with no blocking,
 * fusion or reordering, so that it can be checked against the method by eye.
 * Compiled with -ffp-contract=off so that a*b+c is never fused behind our back.
 */
#include "hf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplications, a key
 * schedule bumped by the Weyl constants between rounds.
 * ------------------------------------------------------------------------- */
void hfo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* key increments    */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint32_t site, uint32_t chain, uint32_t sweep, uint32_t l,
                 uint32_t out[4])
{
    uint32_t ctr[4] = { sweep, l, chain, site };
    uint32_t key[2] = { (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32) };
    hfo_philox4x32_10(ctr, key, out);
}

double hfo_uniform(uint64_t seed, uint32_t site, uint32_t chain, uint32_t sweep, uint32_t l)
{
    uint32_t x[4];
    draw(seed, site, chain, sweep, l, x);
    uint64_t bits = (((uint64_t)x[0] << 32) | (uint64_t)x[1]) >> 11;   /* 53 bits */
    return (double)bits * (1.0 / 9007199254740992.0);                  /* * 2^-53 */
}

void hfo_init_fields(uint64_t seed, uint32_t site, uint32_t chain, int L, int8_t* s)
{
    for (int l = 0; l < L; ++l) {
        uint32_t x[4];
        draw(seed, site, chain, 0xFFFFFFFFu, (uint32_t)l, x);
        s[l] = (x[0] >> 31) ? (int8_t)-1 : (int8_t)1;
    }
}

/* ---------------------------------------------------------------------------
 * Trotter step and Hubbard-Stratonovich coupling: dtau = beta / L,
 * cosh(lambda) = exp(dtau U / 2).
 * ------------------------------------------------------------------------- */
void hfo_constants(double beta, double U, int L, double* dtau, double* lambda)
{
    *dtau = beta / (double)L;
    *lambda = acosh(exp(*dtau * U / 2.0));
}

/* ---------------------------------------------------------------------------
 * Bath matrix g0[l][l'] = g0(tau_l - tau_l'), antiperiodic: g0(tau - beta) = -g0(tau).
 * ------------------------------------------------------------------------- */
void hfo_build_g0(int L, const double* gt, double* g0)
{
    for (int l = 0; l < L; ++l)
        for (int lp = 0; lp < L; ++lp) {
            int d = l - lp;
            if (d >= 0) g0[l * L + lp] = gt[d];
            else        g0[l * L + lp] = -gt[d + L];
        }
}

/* ---------------------------------------------------------------------------
 * Dyson relation G = [1 + (1 - g0)(e^V - 1)]^{-1} g0,  V_l = lambda sigma s_l.
 * Plain Gaussian elimination with partial pivoting on [A | g0].
 * ------------------------------------------------------------------------- */
int hfo_dyson(int L, const double* g0, const int8_t* s, int sigma, double lambda,
              double* G, double* det)
{
    double* A = (double*)malloc(sizeof(double) * (size_t)L * (size_t)L);
    double* B = (double*)malloc(sizeof(double) * (size_t)L * (size_t)L);
    if (!A || !B) { free(A); free(B); return -1; }

    /* A[i][j] = delta_ij + (delta_ij - g0[i][j]) * (exp(V_j) - 1) */
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            double ev = exp(lambda * (double)sigma * (double)s[j]) - 1.0;
            double one = (i == j) ? 1.0 : 0.0;
            A[i * L + j] = one + (one - g0[i * L + j]) * ev;
            B[i * L + j] = g0[i * L + j];
        }

    double d = 1.0;
    for (int k = 0; k < L; ++k) {
        int piv = k;
        double best = fabs(A[k * L + k]);
        for (int i = k + 1; i < L; ++i)
            if (fabs(A[i * L + k]) > best) { best = fabs(A[i * L + k]); piv = i; }
        if (best == 0.0) { free(A); free(B); return -1; }
        if (piv != k) {
            for (int j = 0; j < L; ++j) {
                double t = A[k * L + j]; A[k * L + j] = A[piv * L + j]; A[piv * L + j] = t;
                t = B[k * L + j]; B[k * L + j] = B[piv * L + j]; B[piv * L + j] = t;
            }
            d = -d;
        }
        d *= A[k * L + k];
        for (int i = k + 1; i < L; ++i) {
            double f = A[i * L + k] / A[k * L + k];
            for (int j = k; j < L; ++j) A[i * L + j] -= f * A[k * L + j];
            for (int j = 0; j < L; ++j) B[i * L + j] -= f * B[k * L + j];
        }
    }
    /* back substitution, one right-hand side column at a time */
    for (int c = 0; c < L; ++c)
        for (int i = L - 1; i >= 0; --i) {
            double acc = B[i * L + c];
            for (int j = i + 1; j < L; ++j) acc -= A[i * L + j] * G[j * L + c];
            G[i * L + c] = acc / A[i * L + i];
        }
    if (det) *det = d;
    free(A);
    free(B);
    return 0;
}

/* ---------------------------------------------------------------------------
 * One sweep: for l = 0..L-1, propose s_l -> -s_l.
 *   a_sigma = exp(-2 lambda sigma s_l) - 1
 *   R_sigma = 1 + (1 - G_sigma[l][l]) a_sigma
 *   accept iff u < R_up R_dn
 *   G_sigma <- G_sigma + (a_sigma / R_sigma) (G_sigma[:, l] - e_l) G_sigma[l, :]
 * ------------------------------------------------------------------------- */
static void rank1_update(int L, int l, double a, double R, double* G, double* col, double* row)
{
    for (int i = 0; i < L; ++i) col[i] = G[i * L + l] - ((i == l) ? 1.0 : 0.0);
    for (int j = 0; j < L; ++j) row[j] = G[l * L + j];
    double f = a / R;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j)
            G[i * L + j] += f * col[i] * row[j];
}

double hfo_ratio(int L, double lambda, const int8_t* s, int l, const double* Gup,
                 const double* Gdn, double* a, double* R)
{
    for (int sp = 0; sp < 2; ++sp) {
        double sigma = (sp == 0) ? 1.0 : -1.0;
        const double* G = (sp == 0) ? Gup : Gdn;
        a[sp] = exp(-2.0 * lambda * sigma * (double)s[l]) - 1.0;
        R[sp] = 1.0 + (1.0 - G[l * L + l]) * a[sp];
    }
    return R[0] * R[1];
}

/* Near-tie watch (instrumentation only, no effect on any result): proposals whose uniform lies
 * within tie_rel * |R_up R_dn| of the Metropolis threshold, where two implementations that
 * round differently could decide differently. */
static double tie_rel = 0.0;
static long tie_count = 0;

void hfo_tie_watch(double rel)
{
    tie_rel = rel;
    tie_count = 0;
}

long hfo_tie_count(void) { return tie_count; }

int hfo_sweep(int L, double lambda, uint64_t seed, uint32_t site, uint32_t chain,
              uint32_t sweep, int8_t* s, double* Gup, double* Gdn)
{
    double* col = (double*)malloc(sizeof(double) * (size_t)L);
    double* row = (double*)malloc(sizeof(double) * (size_t)L);
    int accepted = 0;
    for (int l = 0; l < L; ++l) {
        double u = hfo_uniform(seed, site, chain, sweep, (uint32_t)l);
        double a[2], R[2];
        double p = hfo_ratio(L, lambda, s, l, Gup, Gdn, a, R);
        double a_up = a[0], a_dn = a[1], R_up = R[0], R_dn = R[1];
        if (tie_rel > 0.0 && fabs(u - p) < tie_rel * fabs(p)) ++tie_count;
        if (u < p) {
            rank1_update(L, l, a_up, R_up, Gup, col, row);
            rank1_update(L, l, a_dn, R_dn, Gdn, col, row);
            s[l] = (int8_t)(-s[l]);
            ++accepted;
        }
    }
    free(col);
    free(row);
    return accepted;
}

/* ---------------------------------------------------------------------------
 * Measurement: translation-averaged G(tau_m), densities and double occupancy.
 * For a fixed field configuration the two spins are independent, so the
 * equal-time double occupancy of slice l is n_up,l * n_dn,l.
 * ------------------------------------------------------------------------- */
void hfo_measure(int L, const double* Gup, const double* Gdn, double* acc)
{
    const double* G[2] = { Gup, Gdn };
    for (int sp = 0; sp < 2; ++sp)
        for (int m = 0; m < L; ++m) {
            double sum = 0.0;
            for (int l = 0; l < L; ++l) {
                int r = l + m;
                if (r < L) sum += G[sp][r * L + l];
                else       sum -= G[sp][(r - L) * L + l];
            }
            acc[sp * L + m] += sum / (double)L;
        }
    double nup = 0.0, ndn = 0.0, dbl = 0.0;
    for (int l = 0; l < L; ++l) {
        double a = 1.0 - Gup[l * L + l];
        double b = 1.0 - Gdn[l * L + l];
        nup += a;
        ndn += b;
        dbl += a * b;
    }
    acc[2 * L + 0] += nup / (double)L;
    acc[2 * L + 1] += ndn / (double)L;
    acc[2 * L + 2] += dbl / (double)L;
}

long hfo_run_chain(int L, double lambda, const double* g0up, const double* g0dn,
                   uint64_t seed, uint32_t site, uint32_t chain, uint32_t* nsw,
                   int n_warmup, int n_measure, int refresh_every, int refresh_stagger,
                   int bin_size, int8_t* s, double* Gup, double* Gdn, double* bins)
{
    long accepted = 0;
    const int W = 2 * L + 3;
    uint32_t phase = 0u;
    if (refresh_every > 0 && refresh_stagger)
        phase = (site + chain) % (uint32_t)refresh_every;
    for (int k = 0; k < n_warmup + n_measure; ++k) {
        accepted += hfo_sweep(L, lambda, seed, site, chain, *nsw, s, Gup, Gdn);
        *nsw += 1u;
        if (refresh_every > 0 && ((*nsw + phase) % (uint32_t)refresh_every) == 0u) {
            if (hfo_dyson(L, g0up, s, +1, lambda, Gup, 0) != 0) return -1;
            if (hfo_dyson(L, g0dn, s, -1, lambda, Gdn, 0) != 0) return -1;
        }
        if (k >= n_warmup) {
            int b = (k - n_warmup) / bin_size;
            hfo_measure(L, Gup, Gdn, bins + (size_t)b * (size_t)W);
        }
    }
    return accepted;
}

/* ---------------------------------------------------------------------------
 * Exact enumeration: <O> = sum_s w(s) O(G(s)) / sum_s w(s), w(s) = prod_sigma det A_sigma(s).
 * ------------------------------------------------------------------------- */
int hfo_brute_force(int L, double lambda, const double* g0up, const double* g0dn, double* out)
{
    if (L < 1 || L > 20) return -1;
    const int W = 2 * L + 3;
    double* Gup = (double*)malloc(sizeof(double) * (size_t)L * (size_t)L);
    double* Gdn = (double*)malloc(sizeof(double) * (size_t)L * (size_t)L);
    double* one = (double*)calloc((size_t)W, sizeof(double));
    int8_t* s = (int8_t*)malloc((size_t)L);
    for (int k = 0; k < W; ++k) out[k] = 0.0;
    double Z = 0.0;
    int rc = 0;
    for (long cfg = 0; cfg < (1L << L); ++cfg) {
        for (int l = 0; l < L; ++l) s[l] = ((cfg >> l) & 1L) ? (int8_t)-1 : (int8_t)1;
        double dup = 0.0, ddn = 0.0;
        if (hfo_dyson(L, g0up, s, +1, lambda, Gup, &dup) != 0 ||
            hfo_dyson(L, g0dn, s, -1, lambda, Gdn, &ddn) != 0) { rc = -1; break; }
        double w = dup * ddn;
        for (int k = 0; k < W; ++k) one[k] = 0.0;
        hfo_measure(L, Gup, Gdn, one);
        for (int k = 0; k < W; ++k) out[k] += w * one[k];
        Z += w;
    }
    if (rc == 0)
        for (int k = 0; k < W; ++k) out[k] /= Z;
    free(Gup);
    free(Gdn);
    free(one);
    free(s);
    return rc;
}
