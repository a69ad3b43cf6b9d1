// k_qmc_df64.cu -- Hirsch-Fye sweeps with G held as FP32 pairs (sm_103a).
//
// Same method and schedule as the FP64 kernel (one team per Markov chain, G_up/G_dn resident in
// shared memory for all sweeps; per slice: single-flip ratio, Metropolis test, Sherman-Morrison
// update; FP64 Dyson refresh every refresh_every sweeps; measurement into bins), but the state
// and all sweep arithmetic use "double-float" numbers x = hi + lo (two floats, |lo| <= ulp(hi),
// a 48-bit significand), evaluated with error-free transformations on the FP32 pipe:
//   TwoSum (Knuth): s = fl(a + b), e = (a - (s - b')) + (b - b') with b' = s - a, exact a + b = s + e;
//   TwoProd (with FMA): p = fl(a b), e = fma(a, b, -p), exact a b = p + e.
// On GB300 the FP32 pipe retires 72x more FMA than the FP64 pipe, so the Sherman-Morrison update
// (2 L^2 multiply-adds per accepted flip) costs ~12 FP32 instructions per element (the pair is
// renormalised once per sweep, not after every update) instead of one FP64 instruction at 1/64
// of the issue rate.  What stays in FP64: the Dyson refresh (the
// method's re-anchoring step), and the Metropolis test whenever the FP32 estimate of R_up R_dn
// is within its error bound of u -- then the ratio is evaluated in FP64 from the exactly
// representable hi + lo, so every decision is the one FP64 arithmetic takes on the stored G.
// Accuracy: each update adds an absolute error ~2^-47 max|G| (a few times that while lo is
// unnormalised within a sweep); between two refreshes (at most a few hundred updates) this stays
// ~1e-13 of max|G|.
#include "qmc_common.cuh"

namespace hfk {
namespace {

using namespace qmc;

// Shared-memory placement of G[i][j] (8-byte elements, rows of L): for L a power of two the
// column pairs of row i are permuted by XOR with i mod 8, so that a column gather G[i][l],
// i = 0..L-1, spreads over the banks (at most 2-way conflicts instead of 32-way) while every
// column pair stays one aligned 16-byte unit; other L keep the dense order.
template <int L>
constexpr int kSW = ((L & (L - 1)) == 0 && L >= 8) ? ((L / 2 < 8 ? L / 2 : 8) - 1) : 0;
template <int L>
__device__ __forceinline__ int gx(int i, int j) {
    return i * L + ((((j >> 1) ^ (i & kSW<L>)) << 1) | (j & 1));
}

// ------------------------------ double-float arithmetic -------------------------------------
// The _rn intrinsics keep every product and sum separately rounded (no contraction), which the
// error-free transformations rely on.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// x + y with absolute error <= ~2^-47 (|x| + |y|)
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
    const float2 s = two_sum(x.x, y.x);
    return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ float2 df_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
    const float p = __fmul_rn(x.x, y.x);
    float e = fmaf(x.x, y.x, -p);
    e = fmaf(x.x, y.y, e);
    e = fmaf(x.y, y.x, e);
    return fast_two_sum(p, e);
}
// z + x y without the final renormalisation: the Sherman-Morrison updates of a sweep leave lo
// unnormalised (it grows by at most half an ulp of hi per update, so after the <= L updates of
// one sweep |lo| <= (L/2 + 1) ulp(hi) and its own rounding stays ~L 2^-48 |hi|); every element
// is renormalised by df_norm at the end of each sweep, and each diagonal element is
// renormalised before it enters a Metropolis test.
__device__ __forceinline__ float2 df_fma_lazy(float2 x, float2 y, float2 z) {
    const float p = __fmul_rn(x.x, y.x);
    float e = fmaf(x.x, y.x, -p);
    e = fmaf(x.x, y.y, e);
    e = fmaf(x.y, y.x, e);
    const float2 s = two_sum(z.x, p);
    return make_float2(s.x, __fadd_rn(s.y, __fadd_rn(e, z.y)));
}
// hi + lo -> (fl(hi + lo), exact remainder): the same number, normalised
__device__ __forceinline__ float2 df_norm(float2 x) { return two_sum(x.x, x.y); }
// exact double value of a double-float (hi + lo has at most 48 significant bits)
__device__ __forceinline__ double df_to_d(float2 x) {
    return static_cast<double>(x.x) + static_cast<double>(x.y);
}
// split of a double: hi = 23-bit truncation (integer pipe), lo = the remainder
__device__ __forceinline__ float2 d_to_df(double x) {
    const float h = f32_of(x);
    const double hd = (h == 0.0f) ? 0.0 : f64_of(h);
    return make_float2(h, f32_of(x - hd));
}
// 1 / R: FP32 seed (relative error ~2^-23 with R.lo neglected) and one Newton step in
// double-float, which squares the error to ~2^-46.
__device__ __forceinline__ float2 df_recip(float2 R) {
    const float2 one = make_float2(1.0f, 0.0f);
    const float2 r = make_float2(__frcp_rn(R.x), 0.0f);
    const float2 e = df_add(one, df_neg(df_mul(R, r)));
    return df_add(r, df_mul(r, e));
}

// Dyson refresh of both spins in FP64 (as the FP64 kernel: G_sigma = M_sigma^{-1} with
// M_sigma = g0^{-1} e^{V_sigma} - (e^{V_sigma} - 1), dense in the two G buffers), both results
// parked in the chain's global slot, then split into double-floats in the permuted placement.
// check (drift monitor): the outgoing pair state is parked in the global slot first and
// compared with the Dyson solution as that is parked (each thread its own elements).
template <int L, int TW>
__device__ void refresh_both_df(const QmcProblem& P, const TeamSmem<L>& S, int site, double* Gg,
                                int tid, bool check) {
    constexpr int T = 32 * TW;
    float2* X0 = reinterpret_cast<float2*>(S.G0);
    float2* X1 = reinterpret_cast<float2*>(S.G1);
    const GjTeamScratch<L> g(S);
    bool ok = true;
    if (check) {
        for (int e = tid; e < L * L; e += T) {
            const int i = e / L, j = e - (e / L) * L;
            Gg[e] = df_to_d(X0[gx<L>(i, j)]);
            Gg[L * L + e] = df_to_d(X1[gx<L>(i, j)]);
        }
        team_sync<TW>();
    }
    if (P.ev_p == 0.0 && P.ev_m == 0.0) {   // U = 0: G = g0 exactly
        const double* gt = P.gtau + static_cast<size_t>(site) * 2 * L;
        build_bath_matrix<L, TW>(gt, S.G0, tid);
        build_bath_matrix<L, TW>(gt + L, S.G1, tid);
        team_sync<TW>();
    } else {
        const double* gi = P.g0inv + static_cast<size_t>(site) * 2 * L * L;
        build_inverse_dyson<L, TW>(P, gi, S.s, +1, S.G0, tid);
        build_inverse_dyson<L, TW>(P, gi + L * L, S.s, -1, S.G1, tid);
        team_sync<TW>();
        ok = gj_team<L, TW>(S.G0, g.fcol, g.pivrow, g.flag, g.pinv, tid);
        ok = gj_team<L, TW>(S.G1, g.fcol, g.pivrow, g.flag, g.pinv, tid) && ok;
    }
    float v = 0.0f;
    for (int e = tid; e < L * L; e += T) {
        if (check) {
            v = fmaxf(v, static_cast<float>(fabs(S.G0[e] - Gg[e])));
            v = fmaxf(v, static_cast<float>(fabs(S.G1[e] - Gg[L * L + e])));
        }
        Gg[e] = S.G0[e];
        Gg[L * L + e] = S.G1[e];
    }
    if (check) drift_fold(P.drift, v, tid == 0);
    team_sync<TW>();
    for (int e = tid; e < L * L; e += T) {
        const int i = e / L, j = e - (e / L) * L;
        X0[gx<L>(i, j)] = d_to_df(Gg[e]);
        X1[gx<L>(i, j)] = d_to_df(Gg[L * L + e]);
    }
    team_sync<TW>();
    if (!ok && tid == 0) atomicExch(P.status, static_cast<int>(HF_ENUMERIC));
}

// One measurement, accumulated in double-float on the FP32 pipe: the bin accumulator holds pair
// sums of L G(tau_m) and of L n_up, L n_dn, L d (the per-measurement averages times L) in the
// 8-byte slots of bacc; they become doubles, divided by L, only when a bin is written out.  On
// this GPU FP64 instructions do not overlap the pair arithmetic, so the per-sweep path keeps
// none.
__device__ __forceinline__ float2 shfl_xor_df(float2 x, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, x.x, o), __shfl_xor_sync(0xffffffffu, x.y, o));
}

template <int L, int TW>
__device__ void measure_df(const TeamSmem<L>& S, int tid) {
    constexpr int T = 32 * TW;
    const float2* G0 = reinterpret_cast<const float2*>(S.G0);
    const float2* G1 = reinterpret_cast<const float2*>(S.G1);
    float2* acc = reinterpret_cast<float2*>(S.bacc);
    const float2 one = make_float2(1.0f, 0.0f);
    for (int m = tid; m < L; m += T) {
        float2 s0 = make_float2(0.0f, 0.0f), s1 = make_float2(0.0f, 0.0f);
        for (int q = 0; q < L; ++q) {
            int l = q + m;
            if (l >= L) l -= L;
            int r = l + m;
            const bool wrap = r >= L;
            if (wrap) r -= L;
            const float2 x0 = G0[gx<L>(r, l)], x1 = G1[gx<L>(r, l)];
            s0 = df_add(s0, wrap ? df_neg(x0) : x0);
            s1 = df_add(s1, wrap ? df_neg(x1) : x1);
        }
        acc[m] = df_add(acc[m], s0);
        acc[L + m] = df_add(acc[L + m], s1);
    }
    float2 nu = make_float2(0.0f, 0.0f), nd = nu, db = nu;
    for (int l = tid; l < L; l += T) {
        const float2 a = df_add(one, df_neg(df_norm(G0[gx<L>(l, l)])));
        const float2 b = df_add(one, df_neg(df_norm(G1[gx<L>(l, l)])));
        nu = df_add(nu, a);
        nd = df_add(nd, b);
        db = df_add(db, df_mul(a, b));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nu = df_add(nu, shfl_xor_df(nu, o));
        nd = df_add(nd, shfl_xor_df(nd, o));
        db = df_add(db, shfl_xor_df(db, o));
    }
    if constexpr (TW > 1) {
        float2* red = reinterpret_cast<float2*>(S.cr);   // [3][4] pairs
        const int w = tid >> 5;
        if ((tid & 31) == 0) {
            red[w] = nu;
            red[4 + w] = nd;
            red[8 + w] = db;
        }
        team_sync<TW>();
        if (tid == 0) {
            nu = red[0];
            nd = red[4];
            db = red[8];
            for (int w2 = 1; w2 < TW; ++w2) {
                nu = df_add(nu, red[w2]);
                nd = df_add(nd, red[4 + w2]);
                db = df_add(db, red[8 + w2]);
            }
        }
    }
    if (tid == 0) {
        acc[2 * L + 0] = df_add(acc[2 * L + 0], nu);
        acc[2 * L + 1] = df_add(acc[2 * L + 1], nd);
        acc[2 * L + 2] = df_add(acc[2 * L + 2], db);
    }
    team_sync<TW>();
}

// Delayed updates: per spin, the pending columns u_q (stored transposed, Ut[q][i]) and rows
// v_q (V[q][j]) of the accepted flips since the last flush, and the current diagonal.
__host__ __device__ constexpr size_t delayed_bytes(int L, int K) {
    return K > 1 ? static_cast<size_t>(4 * K * L + 2 * L) * sizeof(float2) : 0;
}

// G += sum_q u_q v_q^T in accept order (the same multiply-adds, in the same order, as the
// rank-1 path applies them), then reload the diagonal.
template <int L, int TW>
__device__ void df_flush(float2* G0, float2* G1, const float2* Ut0, const float2* Ut1,
                         const float2* V0, const float2* V1, int m, float2* dg0, float2* dg1,
                         int tid) {
    constexpr int T = 32 * TW;
    if constexpr (T % L == 0) {
        const int j = tid % L;
#pragma unroll 4
        for (int i = tid / L; i < L; i += T / L) {
            float2 a0 = G0[gx<L>(i, j)], a1 = G1[gx<L>(i, j)];
            for (int q = 0; q < m; ++q) {
                a0 = df_fma_lazy(Ut0[q * L + i], V0[q * L + j], a0);
                a1 = df_fma_lazy(Ut1[q * L + i], V1[q * L + j], a1);
            }
            G0[gx<L>(i, j)] = a0;
            G1[gx<L>(i, j)] = a1;
        }
    } else {
        for (int e = tid; e < L * L; e += T) {
            const int i = e / L, j = e - (e / L) * L;
            float2 a0 = G0[gx<L>(i, j)], a1 = G1[gx<L>(i, j)];
            for (int q = 0; q < m; ++q) {
                a0 = df_fma_lazy(Ut0[q * L + i], V0[q * L + j], a0);
                a1 = df_fma_lazy(Ut1[q * L + i], V1[q * L + j], a1);
            }
            G0[gx<L>(i, j)] = a0;
            G1[gx<L>(i, j)] = a1;
        }
    }
    team_sync<TW>();
    for (int i = tid; i < L; i += T) {
        dg0[i] = G0[gx<L>(i, i)];
        dg1[i] = G1[gx<L>(i, i)];
    }
    team_sync<TW>();
}

// Rank-1 update of both spins, G_s[i][j] += u_s[i] v_s[j] with u = cr[0..L) / cr[L..2L) and
// v = cr[2L..3L) / cr[3L..4L).  Each thread takes its elements in groups of up to 8 rows: all
// loads of a group, then the group's arithmetic, then its stores.  The compiler cannot prove
// that the G stores miss the cr loads, so it would otherwise run one element's dependent pair
// arithmetic after another.  For even L a thread owns two adjacent columns: one 128-bit load and
// store per row and spin, and each u[i] serves two elements.
template <int L, int TW>
__device__ __forceinline__ void df_rank1(float2* G0, float2* G1, const float2* cr, int tid) {
    constexpr int T = 32 * TW;
    if constexpr (L % 2 == 0 && T >= L / 2) {
        // column pair (j, j + 1), j = 2 (tid % (L/2)); rows i0, i0 + STEP, ... below L.  STEP =
        // T / (L/2) threads share a pair; the T - STEP L/2 spare threads (L not dividing 2T) sit
        // out.
        constexpr int NCP = L / 2, STEP = T / NCP, NR = (L + STEP - 1) / STEP;
        constexpr int GB8 = NR < 8 ? NR : 8;
        constexpr bool EXACT = (L % STEP == 0) && (NR % GB8 == 0);   // no row guard needed
        constexpr int GB = EXACT ? GB8 : (NR < 4 ? NR : 4);          // guarded rows: fewer live
        if (tid >= STEP * NCP) return;
        const int j = 2 * (tid % NCP), i0 = tid / NCP;
        const float4 r0 = *reinterpret_cast<const float4*>(cr + 2 * L + j);
        const float4 r1 = *reinterpret_cast<const float4*>(cr + 3 * L + j);
        for (int b = 0; b < NR; b += GB) {
            float4 a0[GB], a1[GB];
            float2 c0[GB], c1[GB];
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int i = i0 + (b + k) * STEP;
                if (EXACT || i < L) {
                    a0[k] = *reinterpret_cast<const float4*>(G0 + gx<L>(i, j));
                    a1[k] = *reinterpret_cast<const float4*>(G1 + gx<L>(i, j));
                    c0[k] = cr[i];
                    c1[k] = cr[L + i];
                }
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const float2 x0 = df_fma_lazy(c0[k], make_float2(r0.x, r0.y), make_float2(a0[k].x, a0[k].y));
                const float2 y0 = df_fma_lazy(c0[k], make_float2(r0.z, r0.w), make_float2(a0[k].z, a0[k].w));
                const float2 x1 = df_fma_lazy(c1[k], make_float2(r1.x, r1.y), make_float2(a1[k].x, a1[k].y));
                const float2 y1 = df_fma_lazy(c1[k], make_float2(r1.z, r1.w), make_float2(a1[k].z, a1[k].w));
                a0[k] = make_float4(x0.x, x0.y, y0.x, y0.y);
                a1[k] = make_float4(x1.x, x1.y, y1.x, y1.y);
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int i = i0 + (b + k) * STEP;
                if (EXACT || i < L) {
                    *reinterpret_cast<float4*>(G0 + gx<L>(i, j)) = a0[k];
                    *reinterpret_cast<float4*>(G1 + gx<L>(i, j)) = a1[k];
                }
            }
        }
    } else {
        // elements e = tid + n T, n = 0 .. NE-1 (the last group ragged)
        constexpr int NE = (L * L + T - 1) / T, GB = NE < 8 ? NE : 8;
        for (int b = 0; b < NE; b += GB) {
            float2 a0[GB], a1[GB], c0[GB], c1[GB], v0[GB], v1[GB];
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int e = tid + (b + k) * T;
                if (e < L * L) {
                    const int i = e / L, j = e - (e / L) * L;
                    a0[k] = G0[gx<L>(i, j)];
                    a1[k] = G1[gx<L>(i, j)];
                    c0[k] = cr[i];
                    c1[k] = cr[L + i];
                    v0[k] = cr[2 * L + j];
                    v1[k] = cr[3 * L + j];
                }
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                if (tid + (b + k) * T < L * L) {
                    a0[k] = df_fma_lazy(c0[k], v0[k], a0[k]);
                    a1[k] = df_fma_lazy(c1[k], v1[k], a1[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < GB; ++k) {
                const int e = tid + (b + k) * T;
                if (e < L * L) {
                    const int i = e / L, j = e - (e / L) * L;
                    G0[gx<L>(i, j)] = a0[k];
                    G1[gx<L>(i, j)] = a1[k];
                }
            }
        }
    }
}

// DLY: delayed rank-k updates (P.delay_k > 1); the rank-1 instantiation carries none of their
// buffers or branches.
template <int L, int TW, bool DLY>
__device__ void df_chain(const QmcProblem& P, int c, unsigned char* base, int tid) {
    constexpr int T = 32 * TW;
    constexpr int LL = L * L;
    constexpr int W = 2 * L + 3;
    const TeamSmem<L> S(base);
    float2* G0 = reinterpret_cast<float2*>(S.G0);
    float2* G1 = reinterpret_cast<float2*>(S.G1);
    float2* cr = reinterpret_cast<float2*>(S.cr);
    const int site = c / P.cps;
    const int ch = c - site * P.cps;
    double* Gg = P.G + static_cast<size_t>(c) * 2 * LL;   // 8 bytes per element, pairs here
    float2* Gp = reinterpret_cast<float2*>(Gg);
    const uint2 key = make_uint2(P.seed_lo, P.seed_hi);
    const float2 a_p = make_float2(P.af_p, P.afl_p), a_m = make_float2(P.af_m, P.afl_m);
    const float2 one = make_float2(1.0f, 0.0f);
    const int K = DLY ? P.delay_k : 1;
    float2* Ut0 = reinterpret_cast<float2*>(base + team_bytes(L));   // [K][L]
    float2* Ut1 = Ut0 + K * L;
    float2* V0 = Ut1 + K * L;                                         // [K][L]
    float2* V1 = V0 + K * L;
    float2* dg0 = V1 + K * L;                                         // [L]
    float2* dg1 = dg0 + L;

#ifdef HF_DEBUG_SMEM
    {   // self-check: this team's region [base, base + team + delayed) inside the dynamic window
        extern __shared__ __align__(16) unsigned char smem[];
        unsigned dyn;
        asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const long off = base - smem;
        const long end = off + static_cast<long>(team_bytes(L) + delayed_bytes(L, P.delay_k));
        if (off < 0 || end > static_cast<long>(dyn) || (off & 15) != 0) {
            if (tid == 0) {
                atomicExch(P.status + 2, __LINE__);
                atomicExch(P.status + 3, static_cast<int>(end));
                atomicExch(P.status, static_cast<int>(HF_EINVAL));
            }
            return;
        }
    }
#endif
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
        reinterpret_cast<float2*>(S.bacc)[k] =
            d_to_df((cur_bin < P.max_bins) ? bins_c[static_cast<size_t>(cur_bin) * W + k] * L : 0.0);
    team_sync<TW>();
    if (P.refresh_first) {
        refresh_both_df<L, TW>(P, S, site, Gg, tid, false);   // the bath may have changed
    } else {
        for (int e = tid; e < LL; e += T) {
            const int i = e / L, j = e - (e / L) * L;
            G0[gx<L>(i, j)] = Gp[e];
            G1[gx<L>(i, j)] = Gp[LL + e];
        }
        team_sync<TW>();
    }

    const int nsweeps = P.n_warmup + P.n_measure;
    for (int k = 0; k < nsweeps; ++k) {
        for (int l = tid; l < L; l += T)
            S.ub[l] = uniform_bits53(philox4x32_10(make_uint4(nsw, static_cast<uint32_t>(l),
                                                              static_cast<uint32_t>(ch),
                                                              static_cast<uint32_t>(P.site0 + site)), key));
        int m = 0;                  // pending delayed updates
        if constexpr (DLY)
            for (int i = tid; i < L; i += T) {
                dg0[i] = G0[gx<L>(i, i)];
                dg1[i] = G1[gx<L>(i, i)];
            }
        team_sync<TW>();
        for (int l = 0; l < L; ++l) {
            const float2 g0 = df_norm(DLY ? dg0[l] : G0[gx<L>(l, l)]);
            const float2 g1 = df_norm(DLY ? dg1[l] : G1[gx<L>(l, l)]);
            const int sl = S.s[l];
            const float auf = (sl > 0) ? P.af_p : P.af_m;   // up:   sigma s_l = +s_l
            const float adf = (sl > 0) ? P.af_m : P.af_p;   // down: sigma s_l = -s_l
            // FP32 estimate of the Metropolis test with the error bound of the FP64 kernel
            // (the pair's hi part is within 2^-24 of its value, inside the 2^-23 term)
            const unsigned long long ubits = S.ub[l];
            const float uf = static_cast<float>(static_cast<unsigned>(ubits >> 29)) * 0x1p-24f;
            const float Ruf = fmaf(1.0f - g0.x, auf, 1.0f);
            const float Rdf = fmaf(1.0f - g1.x, adf, 1.0f);
            const float pf = Ruf * Rdf;
            const float eRu = 0x1p-21f * (fabsf(auf) * (fabsf(1.0f - g0.x) + fabsf(g0.x) + 1.0f) + fabsf(Ruf));
            const float eRd = 0x1p-21f * (fabsf(adf) * (fabsf(1.0f - g1.x) + fabsf(g1.x) + 1.0f) + fabsf(Rdf));
            const float guard = 2.0f * (eRu * (fabsf(Rdf) + eRd) + fabsf(Ruf) * eRd +
                                        0x1p-24f * (fabsf(pf) + 1.0f));
            bool accept;
            if (fabsf(uf - pf) > guard) {
                accept = uf < pf;
                if (!(pf > 0.0f) && tid == 0) atomicAdd(P.status + 1, 1);
            } else {
                const double au = (sl > 0) ? P.a_p : P.a_m;
                const double ad = (sl > 0) ? P.a_m : P.a_p;
                const double Ru = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -df_to_d(g0)), au));
                const double Rd = __dadd_rn(1.0, __dmul_rn(__dadd_rn(1.0, -df_to_d(g1)), ad));
                const double p = __dmul_rn(Ru, Rd);
                if (!(p > 0.0) && tid == 0) atomicAdd(P.status + 1, 1);
                accept = static_cast<double>(ubits) * 0x1p-53 < p;
            }
            if (accept) {
                // f_sigma = a_sigma / R_sigma in double-float
                // lanes 0-15 take spin up, lanes 16-31 spin down (the same arithmetic for both,
                // half the instructions), then every lane reads both from the warp
                const bool dn = (tid & 16) != 0;
                const float2 as = (sl > 0) != dn ? a_p : a_m;
                const float2 Rs = df_add(one, df_mul(df_add(one, df_neg(dn ? g1 : g0)), as));
                const float2 fs = df_mul(as, df_recip(Rs));
                const float2 fu = make_float2(__shfl_sync(0xffffffffu, fs.x, 0),
                                              __shfl_sync(0xffffffffu, fs.y, 0));
                const float2 fd = make_float2(__shfl_sync(0xffffffffu, fs.x, 16),
                                              __shfl_sync(0xffffffffu, fs.y, 16));
                if constexpr (DLY) {
#ifdef HF_DEBUG_SMEM
                    if (m < 0 || m >= K) {   // self-check: append slot inside the buffers
                        if (tid == 0) {
                            atomicExch(P.status + 2, __LINE__);
                            atomicExch(P.status + 3, m);
                            atomicExch(P.status, static_cast<int>(HF_EINVAL));
                        }
                        m = 0;
                    }
#endif
                    // every thread of the team has read dg[l] for this decision before any
                    // diagonal or pending slot is written (threads run ahead through rejections)
                    team_sync<TW>();
                    // current column l and row l = stale values + pending products, in accept
                    // order; append u = f (G[:, l] - e_l), v = G[l, :]; update the diagonal
                    for (int i = tid; i < L; i += T) {
                        float2 c0 = G0[gx<L>(i, l)], c1 = G1[gx<L>(i, l)];
                        float2 r0 = G0[gx<L>(l, i)], r1 = G1[gx<L>(l, i)];
                        for (int q = 0; q < m; ++q) {
                            c0 = df_fma_lazy(Ut0[q * L + i], V0[q * L + l], c0);
                            c1 = df_fma_lazy(Ut1[q * L + i], V1[q * L + l], c1);
                            r0 = df_fma_lazy(Ut0[q * L + l], V0[q * L + i], r0);
                            r1 = df_fma_lazy(Ut1[q * L + l], V1[q * L + i], r1);
                        }
                        if (i == l) {
                            c0 = df_add(c0, df_neg(one));
                            c1 = df_add(c1, df_neg(one));
                        }
                        const float2 u0 = df_mul(fu, c0), u1 = df_mul(fd, c1);
                        Ut0[m * L + i] = u0;
                        Ut1[m * L + i] = u1;
                        V0[m * L + i] = r0;
                        V1[m * L + i] = r1;
                        dg0[i] = df_fma_lazy(u0, r0, dg0[i]);
                        dg1[i] = df_fma_lazy(u1, r1, dg1[i]);
                    }
                    team_sync<TW>();
                    if (tid == 0) S.s[l] = static_cast<int8_t>(-sl);
                    ++acc;
                    if (++m == K) {
                        df_flush<L, TW>(G0, G1, Ut0, Ut1, V0, V1, m, dg0, dg1, tid);
                        m = 0;
                    }
                } else {
                    for (int i = tid; i < L; i += T) {
                        float2 x0 = G0[gx<L>(i, l)], x1 = G1[gx<L>(i, l)];
                        if (i == l) {
                            x0 = df_add(x0, df_neg(one));
                            x1 = df_add(x1, df_neg(one));
                        }
                        cr[i] = df_mul(fu, x0);
                        cr[L + i] = df_mul(fd, x1);
                        cr[2 * L + i] = G0[gx<L>(l, i)];
                        cr[3 * L + i] = G1[gx<L>(l, i)];
                    }
                    team_sync<TW>();
                    df_rank1<L, TW>(G0, G1, cr, tid);
                    team_sync<TW>();
                    if (tid == 0) S.s[l] = static_cast<int8_t>(-sl);
                    ++acc;
                }
            }
        }
        if constexpr (DLY) {
            if (m > 0) df_flush<L, TW>(G0, G1, Ut0, Ut1, V0, V1, m, dg0, dg1, tid);
        }
        // renormalise every element after the sweep's lazy updates (threads may still be reading
        // diagonals of the last proposals until the barrier)
        team_sync<TW>();
        for (int e = tid; e < LL; e += T) {
            const int i = e / L, j = e - (e / L) * L;
            G0[gx<L>(i, j)] = df_norm(G0[gx<L>(i, j)]);
            G1[gx<L>(i, j)] = df_norm(G1[gx<L>(i, j)]);
        }
        ++nsw;
        team_sync<TW>();
        if (P.refresh_every > 0 && ((nsw + rphase) % static_cast<uint32_t>(P.refresh_every)) == 0u)
            refresh_both_df<L, TW>(P, S, site, Gg, tid, P.drift != nullptr);
        if (k >= P.n_warmup) {
            measure_df<L, TW>(S, tid);
            ++nmeas;
            if (nmeas % static_cast<uint32_t>(P.bin_size) == 0u) {
                const int b = static_cast<int>(nmeas / P.bin_size) - 1;
                for (int q = tid; q < W; q += T) {
                    float2* acc = reinterpret_cast<float2*>(S.bacc);
                    if (b < P.max_bins) bins_c[static_cast<size_t>(b) * W + q] = df_to_d(acc[q]) / L;
                    acc[q] = make_float2(0.0f, 0.0f);
                }
                team_sync<TW>();
            }
        }
    }

    cur_bin = static_cast<int>(nmeas / P.bin_size);
    for (int q = tid; q < W; q += T)
        if (cur_bin < P.max_bins)
            bins_c[static_cast<size_t>(cur_bin) * W + q] = df_to_d(reinterpret_cast<float2*>(S.bacc)[q]) / L;
    for (int e = tid; e < LL; e += T) {
        const int i = e / L, j = e - (e / L) * L;
        Gp[e] = G0[gx<L>(i, j)];
        Gp[LL + e] = G1[gx<L>(i, j)];
    }
    for (int l = tid; l < L; l += T) P.s[static_cast<size_t>(c) * L + l] = S.s[l];
    if (tid == 0) {
        P.nsw[c] = nsw;
        P.nmeas[c] = nmeas;
        P.acc[c] += acc;
    }
}

template <int L, int TW>
__device__ void run_team_df(const QmcProblem& P, int blk, unsigned char* smem) {
    constexpr int per_block = kBlock / (32 * TW);
    const int team = static_cast<int>(threadIdx.x) / (32 * TW);
    const int slot = blk * per_block + team;
    const long long m = P.slot_mult > 0 ? P.slot_mult : 1;
    const int c = static_cast<int>(slot * m % P.nchain);
    const size_t stride = team_bytes(L) + delayed_bytes(L, P.delay_k);
    if (slot >= P.nchain) return;
    const int tid = static_cast<int>(threadIdx.x) % (32 * TW);
    if constexpr (TW == 1) {   // delayed updates run with one warp per chain
        if (P.delay_k > 1) {
            df_chain<L, TW, true>(P, c, smem + team * stride, tid);
            return;
        }
    }
    df_chain<L, TW, false>(P, c, smem + team * stride, tid);
}

template <int L>
__device__ void run_block_df(const QmcProblem& P, int blk, unsigned char* smem) {
    const int tw = P.team_warps;
    if constexpr (L <= 32) {
        if (tw == 1) run_team_df<L, 1>(P, blk, smem);
        else if (tw == 2) run_team_df<L, 2>(P, blk, smem);
        else run_team_df<L, 4>(P, blk, smem);
    } else {
        if (tw == 2) run_team_df<L, 2>(P, blk, smem);
        else run_team_df<L, 4>(P, blk, smem);
    }
}

__global__ void __launch_bounds__(kBlock, 3) qmc_df64_kernel(const __grid_constant__ QmcBatch B) {
    extern __shared__ __align__(16) unsigned char smem[];
    int pi = 0;
    while (pi + 1 < B.nprob && static_cast<int>(blockIdx.x) >= B.p[pi + 1].block0) ++pi;
    const QmcProblem& P = B.p[pi];
    const int blk = static_cast<int>(blockIdx.x) - P.block0;
    switch (P.L) {
        case 8: run_block_df<8>(P, blk, smem); break;
        case 12: run_block_df<12>(P, blk, smem); break;
        case 16: run_block_df<16>(P, blk, smem); break;
        case 20: run_block_df<20>(P, blk, smem); break;
        case 24: run_block_df<24>(P, blk, smem); break;
        case 32: run_block_df<32>(P, blk, smem); break;
        case 40: run_block_df<40>(P, blk, smem); break;
        case 48: run_block_df<48>(P, blk, smem); break;
        case 64: run_block_df<64>(P, blk, smem); break;
        default: break;
    }
}

}  // namespace

size_t qmc_df64_smem_bytes(int L, int team_warps, int delay_k) {
    return static_cast<size_t>(4 / team_warps) * (team_bytes(L) + delayed_bytes(L, delay_k));
}

cudaError_t launch_qmc_df64(const QmcBatch& b, size_t smem, cudaStream_t st) {
    // the largest block (two-warp teams at L = 64) needs ~136 KB; set what this launch asks for
    cudaError_t e = cudaFuncSetAttribute(qmc_df64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (b.nblocks <= 0) return cudaSuccess;
    qmc_df64_kernel<<<b.nblocks, kBlock, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace hfk
