// k_qmc_f64.cu -- FP64 Hirsch-Fye QMC sweeps, resident in shared memory (sm_103a).
//
// One "team" (one warp for L <= 32, the whole 4-warp block for L > 32) owns one Markov chain
// for the whole launch: its G_up, G_dn (L x L, FP64) stay in shared memory through
// n_warmup + n_measure sweeps.  Per slice l of a sweep ("Model and Methods": Hirsch-Fye at
// fixed dtau, with the single-flip ratio, Metropolis acceptance and Sherman-Morrison update):
//     R_sigma = 1 + (1 - G_sigma[l][l]) (e^{-2 lambda sigma s_l} - 1),  accept iff u < R_up R_dn,
//     G_sigma += (a_sigma / R_sigma) (G_sigma[:, l] - e_l) G_sigma[l, :].
// The Dyson refresh G = [1 + (1 - g0)(e^V - 1)]^{-1} g0 runs after every refresh_every-th sweep
// of the chain, as G = M^{-1} with M = g0^{-1} e^V - (e^V - 1) (the same relation multiplied
// out): M is built from the site's g0^{-1} (computed once per bath by g0inv_kernel below, from
// the antiperiodic bath matrix g0[l][l'] = g~0(tau_l - tau_l')) and inverted in place by
// Gauss-Jordan elimination with partial pivoting in shared memory.  Measured sweeps accumulate
// G(tau_m), n_sigma and the double occupancy into the chain's current bin.
//
// GB300 has ~1 TFLOP/s of FP64 (DFMA and DMMA alike, 72x below FFMA), so this kernel is bound
// by the FP64 pipe; it keeps the pipe busy with 12 chains per SM and issues no FP64 work that
// the method does not need (the index arithmetic stays on the integer pipe).
#include <algorithm>

#include "qmc_common.cuh"

namespace hfk {
namespace {

using namespace qmc;


// Dyson refresh of both spins: G_sigma = M_sigma^{-1}, M_sigma = g0^{-1} e^{V_sigma} -
// (e^{V_sigma} - 1) built from the site's g0^{-1} and inverted in place in G_sigma's buffer.
template <int L, int TW>
__device__ void refresh_both(const QmcProblem& P, const TeamSmem<L>& S, int site, int tid) {
    if (P.ev_p == 0.0 && P.ev_m == 0.0) {   // U = 0
        const double* gt = P.gtau + static_cast<size_t>(site) * 2 * L;
        build_bath_matrix<L, TW>(gt, S.G0, tid);
        build_bath_matrix<L, TW>(gt + L, S.G1, tid);
        team_sync<TW>();
        return;
    }
    const GjTeamScratch<L> g(S);
    const double* gi = P.g0inv + static_cast<size_t>(site) * 2 * L * L;
    build_inverse_dyson<L, TW>(P, gi, S.s, +1, S.G0, tid);
    build_inverse_dyson<L, TW>(P, gi + L * L, S.s, -1, S.G1, tid);
    team_sync<TW>();
    bool ok = gj_team<L, TW>(S.G0, g.fcol, g.pivrow, g.flag, g.pinv, tid);
    ok = gj_team<L, TW>(S.G1, g.fcol, g.pivrow, g.flag, g.pinv, tid) && ok;
    if (!ok && tid == 0) atomicExch(P.status, static_cast<int>(HF_ENUMERIC));
}

// Rank-1 update of both spins, G_s[i][j] += u_s[i] v_s[j] (u = cr[0..L) / cr[L..2L),
// v = cr[2L..3L) / cr[3L..4L)), one DFMA per element.  Each thread takes its elements in groups
// -- all loads, then the DFMAs, then the stores -- because the compiler cannot prove that the G
// stores miss the cr loads and would otherwise serialise the elements.
template <int L, int TW>
__device__ __forceinline__ void rank1(double* G0, double* G1, const double* cr, int tid) {
    constexpr int T = 32 * TW;
    if constexpr (T % L == 0) {
        // one column j per thread (its row entries stay in registers); rows i0, i0 + STEP, ...
        constexpr int STEP = T / L, NR = (L + STEP - 1) / STEP, GB = NR < 8 ? NR : 8;
        const int j = tid % L, i0 = tid / L;
        if (STEP > L && i0 >= L) return;
        const double r0 = cr[2 * L + j], r1 = cr[3 * L + j];
        for (int b = 0; b < NR; b += GB) {
            double a0[GB], a1[GB], c0[GB], c1[GB];
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int i = i0 + (b + k) * STEP;
                a0[k] = G0[i * L + j];
                a1[k] = G1[i * L + j];
                c0[k] = cr[i];
                c1[k] = cr[L + i];
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                a0[k] = fma(c0[k], r0, a0[k]);
                a1[k] = fma(c1[k], r1, a1[k]);
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int i = i0 + (b + k) * STEP;
                G0[i * L + j] = a0[k];
                G1[i * L + j] = a1[k];
            }
        }
    } else {
        // elements e = tid + n T (the last group ragged), groups of up to 4 (register budget)
        constexpr int NE = (L * L + T - 1) / T, GB = NE < 4 ? NE : 4;
        for (int b = 0; b < NE; b += GB) {
            double a0[GB], a1[GB], c0[GB], c1[GB], v0[GB], v1[GB];
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int e = tid + (b + k) * T;
                if (e < L * L) {
                    const int i = e / L, j = e - (e / L) * L;
                    a0[k] = G0[e];
                    a1[k] = G1[e];
                    c0[k] = cr[i];
                    c1[k] = cr[L + i];
                    v0[k] = cr[2 * L + j];
                    v1[k] = cr[3 * L + j];
                }
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                if (tid + (b + k) * T < L * L) {
                    a0[k] = fma(c0[k], v0[k], a0[k]);
                    a1[k] = fma(c1[k], v1[k], a1[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int e = tid + (b + k) * T;
                if (e < L * L) {
                    G0[e] = a0[k];
                    G1[e] = a1[k];
                }
            }
        }
    }
}

// Accumulate one measurement into bacc.
template <int L, int TW>
__device__ void measure(const TeamSmem<L>& S, int tid) {
    constexpr int T = 32 * TW;
    // G(tau_m) = (1/L) sum_l sgn G[(l+m) mod L][l]; thread m walks l in a skewed order so that
    // the 32 lanes of a warp hit different banks.
    for (int m = tid; m < L; m += T) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < L; ++q) {
            int l = q + m;
            if (l >= L) l -= L;
            int r = l + m;
            const bool wrap = r >= L;
            if (wrap) r -= L;
            const double x0 = S.G0[r * L + l], x1 = S.G1[r * L + l];
            s0 = wrap ? s0 - x0 : s0 + x0;
            s1 = wrap ? s1 - x1 : s1 + x1;
        }
        S.bacc[m] += s0 / L;
        S.bacc[L + m] += s1 / L;
    }
    double nu = 0.0, nd = 0.0, db = 0.0;
    for (int l = tid; l < L; l += T) {
        const double a = 1.0 - S.G0[l * L + l];
        const double b = 1.0 - S.G1[l * L + l];
        nu += a;
        nd += b;
        db += a * b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nu += __shfl_xor_sync(0xffffffffu, nu, o);
        nd += __shfl_xor_sync(0xffffffffu, nd, o);
        db += __shfl_xor_sync(0xffffffffu, db, o);
    }
    if constexpr (TW > 1) {
        const int w = tid >> 5;
        if ((tid & 31) == 0) {
            S.red[w] = nu;          // red has 8 slots; TW <= 4 uses red[0..3] and cr[0..7]
            S.cr[w] = nd;
            S.cr[4 + w] = db;
        }
        team_sync<TW>();
        if (tid == 0) {
            nu = 0.0;
            nd = 0.0;
            db = 0.0;
            for (int w2 = 0; w2 < TW; ++w2) {
                nu += S.red[w2];
                nd += S.cr[w2];
                db += S.cr[4 + w2];
            }
        }
    }
    if (tid == 0) {
        S.bacc[2 * L + 0] += nu / L;
        S.bacc[2 * L + 1] += nd / L;
        S.bacc[2 * L + 2] += db / L;
    }
    team_sync<TW>();
}

template <int L, int TW>
__device__ void qmc_chain(const QmcProblem& P, int c, unsigned char* base, int tid) {
    constexpr int T = 32 * TW;
    constexpr int LL = L * L;
    constexpr int W = 2 * L + 3;
    const TeamSmem<L> S(base);
    const int site = c / P.cps;
    const int ch = c - site * P.cps;
    double* Gg = P.G + static_cast<size_t>(c) * 2 * LL;
    const uint2 key = make_uint2(P.seed_lo, P.seed_hi);

    for (int l = tid; l < L; l += T) S.s[l] = P.s[static_cast<size_t>(c) * L + l];
    uint32_t nsw = P.nsw[c];
    // refresh phase: with staggering, chain (site, ch) refreshes when nsw + site + ch is a
    // multiple of refresh_every, so the chains sharing an SM do not all wait on the FP64 pipe
    // in the same sweep
    const uint32_t rphase =
        (P.refresh_stagger && P.refresh_every > 0)
            ? (static_cast<uint32_t>(P.site0 + site) + static_cast<uint32_t>(ch)) %
                  static_cast<uint32_t>(P.refresh_every)
            : 0u;
    uint32_t nmeas = P.nmeas[c];
    unsigned long long acc = 0ull;
    int cur_bin = static_cast<int>(nmeas / P.bin_size);
    double* bins_c = P.bins + static_cast<size_t>(c) * P.max_bins * W;
    for (int k = tid; k < W; k += T)
        S.bacc[k] = (cur_bin < P.max_bins) ? bins_c[static_cast<size_t>(cur_bin) * W + k] : 0.0;
    team_sync<TW>();
    if (P.refresh_first) {
        refresh_both<L, TW>(P, S, site, tid);
    } else {
        for (int e = tid; e < LL; e += T) {
            S.G0[e] = Gg[e];
            S.G1[e] = Gg[LL + e];
        }
        team_sync<TW>();
    }

    const int nsweeps = P.n_warmup + P.n_measure;
    for (int k = 0; k < nsweeps; ++k) {
        for (int l = tid; l < L; l += T)
            S.ub[l] = uniform_bits53(philox4x32_10(make_uint4(nsw, static_cast<uint32_t>(l),
                                                              static_cast<uint32_t>(ch),
                                                              static_cast<uint32_t>(P.site0 + site)), key));
        team_sync<TW>();
        for (int l = 0; l < L; ++l) {
            const double g0 = S.G0[l * L + l];
            const double g1 = S.G1[l * L + l];
            const int sl = S.s[l];
            const double au = (sl > 0) ? P.a_p : P.a_m;   // up:   sigma s_l = +s_l
            const double ad = (sl > 0) ? P.a_m : P.a_p;   // down: sigma s_l = -s_l
            const float auf = (sl > 0) ? P.af_p : P.af_m;
            const float adf = (sl > 0) ? P.af_m : P.af_p;
            // Metropolis test u < R_up R_dn.  An FP32 estimate decides whenever |u - p| exceeds
            // twice a bound on its error; otherwise the FP64 product decides.  Either way the
            // outcome is that of the FP64 arithmetic.  Error of the estimate: g truncated to 23
            // bits (2^-23 |g|), 1 - g and a rounded (2^-24), one fused rounding of R (2^-24 |R|)
            // give |R - Rf| <= 2^-21 (|a|(|1-g| + |g| + 1) + |Rf|) =: eR; the product adds
            // eRu (|Rdf| + eRd) + |Ruf| eRd + 2^-24 |pf|, and u carries 2^-24.
            const unsigned long long ubits = S.ub[l];
            const float uf = static_cast<float>(static_cast<unsigned>(ubits >> 29)) * 0x1p-24f;
            const float g0f = f32_of(g0), g1f = f32_of(g1);
            const float Ruf = fmaf(1.0f - g0f, auf, 1.0f);
            const float Rdf = fmaf(1.0f - g1f, adf, 1.0f);
            const float pf = Ruf * Rdf;
            const float eRu = 0x1p-21f * (fabsf(auf) * (fabsf(1.0f - g0f) + fabsf(g0f) + 1.0f) + fabsf(Ruf));
            const float eRd = 0x1p-21f * (fabsf(adf) * (fabsf(1.0f - g1f) + fabsf(g1f) + 1.0f) + fabsf(Rdf));
            const float guard = 2.0f * (eRu * (fabsf(Rdf) + eRd) + fabsf(Ruf) * eRd +
                                        0x1p-24f * (fabsf(pf) + 1.0f));
            bool accept;
            double Ru = 0.0, Rd = 0.0;
            if (fabsf(uf - pf) > guard) {
                accept = uf < pf;
                if (!(pf > 0.0f) && tid == 0) atomicAdd(P.status + 1, 1);
                if (accept) {
                    Ru = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -g0), au));
                    Rd = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -g1), ad));
                }
            } else {
                Ru = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -g0), au));
                Rd = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -g1), ad));
                const double p = __dmul_rn(Ru, Rd);
                if (!(p > 0.0) && tid == 0) atomicAdd(P.status + 1, 1);
                accept = static_cast<double>(ubits) * 0x1p-53 < p;
            }
            if (accept) {
                const double fu = au * recip64(Ru, Ruf);
                const double fd = ad * recip64(Rd, Rdf);
                for (int i = tid; i < L; i += T) {
                    const double one = (i == l) ? 1.0 : 0.0;
                    S.cr[i] = fu * (S.G0[i * L + l] - one);
                    S.cr[L + i] = fd * (S.G1[i * L + l] - one);
                    S.cr[2 * L + i] = S.G0[l * L + i];
                    S.cr[3 * L + i] = S.G1[l * L + i];
                }
                team_sync<TW>();
                rank1<L, TW>(S.G0, S.G1, S.cr, tid);
                team_sync<TW>();
                if (tid == 0) S.s[l] = static_cast<int8_t>(-sl);
                ++acc;
            }
        }
        ++nsw;
        team_sync<TW>();
        if (P.refresh_every > 0 && ((nsw + rphase) % static_cast<uint32_t>(P.refresh_every)) == 0u) {
            if (P.drift) {   // drift monitor: park the updated state in the chain's global slot
                for (int e = tid; e < LL; e += T) {
                    Gg[e] = S.G0[e];
                    Gg[LL + e] = S.G1[e];
                }
                team_sync<TW>();
            }
            refresh_both<L, TW>(P, S, site, tid);
            if (P.drift) {   // ... and compare it with the Dyson solution (each thread its own e)
                float v = 0.0f;
                for (int e = tid; e < LL; e += T) {
                    v = fmaxf(v, static_cast<float>(fabs(S.G0[e] - Gg[e])));
                    v = fmaxf(v, static_cast<float>(fabs(S.G1[e] - Gg[LL + e])));
                }
                drift_fold(P.drift, v, tid == 0);
            }
        }
        if (k >= P.n_warmup) {
            measure<L, TW>(S, tid);
            ++nmeas;
            if (nmeas % static_cast<uint32_t>(P.bin_size) == 0u) {
                const int b = static_cast<int>(nmeas / P.bin_size) - 1;
                for (int q = tid; q < W; q += T) {
                    if (b < P.max_bins) bins_c[static_cast<size_t>(b) * W + q] = S.bacc[q];
                    S.bacc[q] = 0.0;
                }
                team_sync<TW>();
            }
        }
    }

    // write the state back
    cur_bin = static_cast<int>(nmeas / P.bin_size);
    for (int q = tid; q < W; q += T)
        if (cur_bin < P.max_bins) bins_c[static_cast<size_t>(cur_bin) * W + q] = S.bacc[q];
    for (int e = tid; e < LL; e += T) {
        Gg[e] = S.G0[e];
        Gg[LL + e] = S.G1[e];
    }
    for (int l = tid; l < L; l += T) P.s[static_cast<size_t>(c) * L + l] = S.s[l];
    if (tid == 0) {
        P.nsw[c] = nsw;
        P.nmeas[c] = nmeas;
        P.acc[c] += acc;
    }
}

template <int L, int TW>
__device__ void run_team(const QmcProblem& P, int blk, unsigned char* smem) {
    constexpr int per_block = kBlock / (32 * TW);
    const int team = static_cast<int>(threadIdx.x) / (32 * TW);
    const int slot = blk * per_block + team;
    const long long m = P.slot_mult > 0 ? P.slot_mult : 1;
    const int c = static_cast<int>(slot * m % P.nchain);
    if (slot < P.nchain)
        qmc_chain<L, TW>(P, c, smem + team * team_bytes(L), static_cast<int>(threadIdx.x) % (32 * TW));
}

template <int L>
__device__ void run_block(const QmcProblem& P, int blk, unsigned char* smem) {
    const int tw = P.team_warps;
    if constexpr (L <= 32) {
        if (tw == 1) run_team<L, 1>(P, blk, smem);
        else if (tw == 2) run_team<L, 2>(P, blk, smem);
        else run_team<L, 4>(P, blk, smem);
    } else {
        if (tw == 2) run_team<L, 2>(P, blk, smem);
        else run_team<L, 4>(P, blk, smem);
    }
}

__global__ void __launch_bounds__(kBlock, 3) qmc_f64_kernel(const __grid_constant__ QmcBatch B) {
    extern __shared__ __align__(16) unsigned char smem[];
    int pi = 0;
    while (pi + 1 < B.nprob && static_cast<int>(blockIdx.x) >= B.p[pi + 1].block0) ++pi;
    const QmcProblem& P = B.p[pi];
    const int blk = static_cast<int>(blockIdx.x) - P.block0;
    switch (P.L) {
        case 8: run_block<8>(P, blk, smem); break;
        case 12: run_block<12>(P, blk, smem); break;
        case 16: run_block<16>(P, blk, smem); break;
        case 20: run_block<20>(P, blk, smem); break;
        case 24: run_block<24>(P, blk, smem); break;
        case 32: run_block<32>(P, blk, smem); break;
        case 40: run_block<40>(P, blk, smem); break;
        case 48: run_block<48>(P, blk, smem); break;
        case 64: run_block<64>(P, blk, smem); break;
        default: break;
    }
}

__global__ void init_fields_kernel(int8_t* s, int nchain, int cps, int L, uint32_t seed_lo,
                                   uint32_t seed_hi, int site0) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nchain * L) return;
    const int c = idx / L, l = idx - (idx / L) * L;
    const int site = site0 + c / cps, ch = c - (c / cps) * cps;
    const uint4 x = philox4x32_10(make_uint4(0xFFFFFFFFu, static_cast<uint32_t>(l),
                                             static_cast<uint32_t>(ch),
                                             static_cast<uint32_t>(site)),
                                  make_uint2(seed_lo, seed_hi));
    s[idx] = (x.x >> 31) ? static_cast<int8_t>(-1) : static_cast<int8_t>(1);
}

// g0^{-1} of every (site, spin) of every problem of a batch, for the refreshes: one block of
// kBlock threads per (problem, site, spin) builds the antiperiodic bath matrix
// g0[l][l'] = g~0(tau_l - tau_l') (g~0 negated for l < l') and inverts it by Gauss-Jordan.
__host__ __device__ constexpr size_t g0inv_smem(int L) {
    // M[L*L] + fcol[L] + pinv f64, flag[2] + pivrow[L] int
    return static_cast<size_t>(L * L + L + 1) * 8 + static_cast<size_t>(L + 2) * 4;
}

template <int L>
__device__ void g0inv_block(const QmcProblem& P, int b, unsigned char* smem) {
    constexpr int TW = kBlock / 32;
    double* M = reinterpret_cast<double*>(smem);
    double* fcol = M + L * L;
    double* pinv = fcol + L;
    int* flag = reinterpret_cast<int*>(pinv + 1);
    int* pivrow = flag + 2;
    const int tid = threadIdx.x;
    const double* gt = P.gtau + static_cast<size_t>(b) * L;
    for (int e = tid; e < L * L; e += kBlock) {
        const int i = e / L, j = e - (e / L) * L;
        const int d = i - j;
        M[e] = (d >= 0) ? gt[d] : -gt[d + L];
    }
    __syncthreads();
    const bool ok = gj_team<L, TW>(M, fcol, pivrow, flag, pinv, tid);
    double* out = P.g0inv + static_cast<size_t>(b) * L * L;
    for (int e = tid; e < L * L; e += kBlock) out[e] = M[e];
    if (!ok && tid == 0) atomicExch(P.status, static_cast<int>(HF_ENUMERIC));
}

__global__ void __launch_bounds__(kBlock) g0inv_kernel(const __grid_constant__ QmcBatch B) {
    extern __shared__ __align__(16) unsigned char smem[];
    int pi = 0, base = 0;
    while (pi < B.nprob) {
        const int nb = 2 * (B.p[pi].nchain / B.p[pi].cps);
        if (static_cast<int>(blockIdx.x) < base + nb) break;
        base += nb;
        ++pi;
    }
    if (pi >= B.nprob) return;
    const QmcProblem& P = B.p[pi];
    const int b = static_cast<int>(blockIdx.x) - base;
    switch (P.L) {
        case 8: g0inv_block<8>(P, b, smem); break;
        case 12: g0inv_block<12>(P, b, smem); break;
        case 16: g0inv_block<16>(P, b, smem); break;
        case 20: g0inv_block<20>(P, b, smem); break;
        case 24: g0inv_block<24>(P, b, smem); break;
        case 32: g0inv_block<32>(P, b, smem); break;
        case 40: g0inv_block<40>(P, b, smem); break;
        case 48: g0inv_block<48>(P, b, smem); break;
        case 64: g0inv_block<64>(P, b, smem); break;
        case 128: g0inv_block<128>(P, b, smem); break;
        default: break;
    }
}

}  // namespace

cudaError_t launch_g0_inverse(const QmcBatch& b, cudaStream_t st) {
    int blocks = 0;
    size_t smem = 0;
    for (int i = 0; i < b.nprob; ++i) {
        blocks += 2 * (b.p[i].nchain / b.p[i].cps);
        smem = std::max(smem, g0inv_smem(b.p[i].L));
    }
    cudaError_t e = cudaFuncSetAttribute(g0inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(g0inv_smem(128)));
    if (e != cudaSuccess) return e;
    if (blocks <= 0) return cudaSuccess;
    g0inv_kernel<<<blocks, kBlock, smem, st>>>(b);
    return cudaGetLastError();
}

bool qmc_f64_supported(int L) {
    switch (L) {
        case 8: case 12: case 16: case 20: case 24: case 32: case 40: case 48: case 64:
            return true;
        default:
            return false;
    }
}

int qmc_default_team_warps(int L) { return L <= 32 ? 1 : 4; }
int qmc_f64_chains_per_block(int L, int team_warps) { (void)L; return 4 / team_warps; }

size_t qmc_f64_smem_bytes(int L, int team_warps) {
    return static_cast<size_t>(4 / team_warps) * team_bytes(L);
}

cudaError_t launch_qmc_f64(const QmcBatch& b, size_t smem, cudaStream_t st) {
    // the largest block (two-warp teams at L = 64) needs ~136 KB; set what this launch asks for
    cudaError_t e = cudaFuncSetAttribute(qmc_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (b.nblocks <= 0) return cudaSuccess;
    qmc_f64_kernel<<<b.nblocks, kBlock, smem, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_init_fields(int8_t* s, int nchain, int cps, int L, uint32_t seed_lo,
                               uint32_t seed_hi, cudaStream_t st, int site0) {
    const int n = nchain * L;
    if (n <= 0) return cudaSuccess;
    init_fields_kernel<<<(n + 255) / 256, 256, 0, st>>>(s, nchain, cps, L, seed_lo, seed_hi, site0);
    return cudaGetLastError();
}

}  // namespace hfk
