// k_refresh_tc.cu -- FP64 Dyson refresh of the mixed-precision form on the tensor cores (L = 128).
//
// The refresh G = [1 + (1 - g0)(e^V - 1)]^{-1} g0 is the inverse of M = g0^{-1} e^V - (e^V - 1)
// (the Dyson relation multiplied out by g0^{-1}, which is kept per bath).  After an FP32 sweep the
// chain's G is an approximate inverse X0 of M, good to a few parts in 10^5, so two Newton steps
//     R = 1 - M X,   X <- X + X R
// take it to FP64 accuracy: each step squares the relative error, and the products themselves
// must be accurate only to what the step needs.  Step 0 forms the residual from 7-digit operands
// (levels s + t <= 8) and the correction from 5-digit ones (<= 6), which leaves an error small
// enough that one full step (8 digits, levels <= 9; correction as before) converges; a second
// full step runs when it has not.  Every product is formed
// exactly on the tensor cores from base-256 digits (tc_ozaki.cuh), so the FP64 pipe, which GB300
// has cut to 2 multiply-adds per clock per SM, does one addition per element per step instead of
// the L^3 multiply-adds of an elimination.  M X is evaluated as g0^{-1} (E X) - D X with E =
// diag(e^V), D = diag(e^V - 1): the digits of g0^{-1} are cut once per bath, E X is cut per
// refresh on the integer pipe (the significands of e and x multiplied exactly), and D X enters the
// residual in fixed point.
//
// One 256-thread CTA per chain (one per SM: 173 KB of shared memory, all 512 TMEM columns).  A
// product runs in two passes of 64 output columns; per pass, K = 128 in four chunks of 32, double
// buffered: while the tensor cores work on one chunk, all threads cut the digits of the next.
// Thread 0 issues the MMAs (M = 128, N = 64, K = 16; one accumulator per level n = s + t), commits
// them to an mbarrier, and after the last chunk every thread reads its row of each level back
// from TMEM and combines the levels in 64-bit integers.
//
// If the Newton residual does not fall below 2^-24 within two full steps (an FP32 state too far
// from the inverse), or the operands' scales are too large for the residual's accuracy (a badly
// conditioned G) or leave the fixed-point range, the chain is flagged and refreshed by the Gauss-Jordan
// kernel instead (launch_refresh_f64_listed); its outputs here are not written.
#include <algorithm>

#include "k_refresh_tc.cuh"
#include "refresh_measure.cuh"
#include "tc_ozaki.cuh"

namespace hfk {
namespace {

using namespace tc;

constexpr int L = kTcL, LL = L * L;
constexpr int kThreads = 512;
constexpr int KC = 32;              // K per chunk
constexpr int NCH = L / KC;         // chunks
constexpr int SMAX = kTcDigits;
constexpr int A_SL = L * KC * 2;    // bytes of one digit of an A chunk (128 rows x 32 K, bf16)
// a B chunk of NP output columns: NP * KC * 2 bytes per digit; the buffer holds SMAX digits of
// A and SMAX digits of 64 columns, or SMAX / 2 digits of all 128
constexpr int BUFB = SMAX * (A_SL + 64 * KC * 2);
constexpr uint32_t kTmemCols = 512;
constexpr int kConvergedExp = -24;  // Newton residual bound 2^-24: the step's remaining error,
                                    // its square, is below the products' own accuracy
constexpr int kFarExp = -4;         // a first residual above 2^-4: no approximate inverse
// Accuracy limit of the residual: its error is about 2^(-55 + Ta_i + Tb_j) (the operands' 62-bit
// fixed point and the dropped levels), i.e. relative to G about 2^(-55 + max Ta + max Tb) times
// a modest factor.  Chains whose scales exceed this bound -- G with entries in the hundreds, a
// badly conditioned Dyson matrix -- are left to the Gauss-Jordan refresh, so that the tensor-core
// result stays within about 1e-12 of the exact G relative to its largest entry.
constexpr int kMaxScaleSum = 12;

struct Smem {
    unsigned char buf[2][BUFB];     // double-buffered digit chunks: A digits, then B digits
    int rowT[L], colT[L];           // power-of-two scales of the current operands
    int nrowT[L], ncolT[L];         // the next product's, gathered by this product's epilogue
    int gT[L];                      // row scales of g0^{-1} (this spin)
    int tmpT[kThreads];
    unsigned long long red[kThreads / 32];
    int8_t s[L];                    // the chain's fields
    uint64_t mbar[2];               // MMAs of the chunk in buffer b complete
    uint64_t tbar[2];               // bulk copies into buffer b complete
    uint32_t tmem;
    int flag;                       // fallback requested
    int timeout;
};

__device__ __forceinline__ unsigned char* bufA(Smem& S, int b, int s) { return S.buf[b] + s * A_SL; }
template <int NP>
__device__ __forceinline__ unsigned char* bufB(Smem& S, int b, int t) {
    return S.buf[b] + SMAX * A_SL + t * (NP * KC * 2);
}

// significand (with the implicit bit) and exponent of a normal double: x = m 2^(E - 52)
__device__ __forceinline__ void split_double(double x, unsigned long long& m, int& E) {
    const long long b = __double_as_longlong(x);
    m = (static_cast<unsigned long long>(b) & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    E = static_cast<int>((b >> 52) & 0x7FF) - 1023;
}

// D 2^(54 - 8 n) as an integer (levels above 6 lose their lowest bits, rounded)
__device__ __forceinline__ long long level_shift(long long D, int n) {
    const int sh = 54 - 8 * n;
    return sh >= 0 ? (D << sh) : ((D + (1ll << (-sh - 1))) >> (-sh));
}

// max of x over the block (non-negative integers), every thread gets it
__device__ __forceinline__ unsigned long long block_max(Smem& S, unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned long long m = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) m = S.red[w] > m ? S.red[w] : m;
    return m;
}

// ------------------------------------------------------------------------------------------
// operand fills: one K-chunk of every digit, laid out as K-major core matrices
// (core (group, kc) at (group * 4 + kc) * 128 bytes, row r of the core at r * 16)
// ------------------------------------------------------------------------------------------

// A from precomputed digit chunks (each an 8 KB block in exactly this layout): SA bulk copies by
// thread 0, landing on tbar[b]; the MMA issuer waits for them
template <int SA>
__device__ void fill_A_digits(Smem& S, int b, int c, const uint16_t* digits) {
    if (threadIdx.x == 0) {
        mbar_expect_tx(&S.tbar[b], SA * A_SL);
#pragma unroll
        for (int s = 0; s < SA; ++s)
            bulk_copy_g2s(bufA(S, b, s), digits + (static_cast<size_t>(s) * NCH + c) * (A_SL / 2),
                          A_SL, &S.tbar[b]);
    }
}

// NE (4 or 8) fixed-point magnitudes and signs -> SD digit rows of NE bf16 at base + (s - 1) stride
// + off.  Digits top down: d = round(r / 2^(62 - 8 s)) of the remainder r, the eighth digit the last
// 6 bits at weight 2^-64 (digits_of gives the same expansion bottom up).
template <int SD, int NE>
__device__ __forceinline__ void store_digits(const unsigned long long (&U)[NE], const bool (&neg)[NE],
                                             unsigned char* base, int stride, int off) {
    long long r[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) r[q] = static_cast<long long>(U[q]);
#pragma unroll
    for (int s = 1; s <= SD; ++s) {
        int d[NE];
#pragma unroll
        for (int q = 0; q < NE; ++q) {
            if (s < 8) {
                const int sh = 62 - 8 * s;
                const long long v = (r[q] + (1ll << (sh - 1))) >> sh;
                r[q] -= v << sh;
                d[q] = static_cast<int>(v);
            } else {
                d[q] = static_cast<int>(r[q] << 2);
            }
        }
        uint32_t w[NE / 2];
#pragma unroll
        for (int q = 0; q < NE / 2; ++q) w[q] = bf16x2_digits(d[2 * q], d[2 * q + 1], neg[2 * q], neg[2 * q + 1]);
        unsigned char* dst = base + (s - 1) * stride + off;
        if constexpr (NE == 8) *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        else *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
    }
}

// The operand fills of a K-chunk are objects with two steps: load(c) reads the chunk's FP64
// values from global memory into registers, cut(b, c) turns them into digits in buffer b.
// product_pass loads chunk c + 1 right after cutting chunk c, so the global reads are in flight
// during the barrier, the MMA issue and the wait for the next buffer.

// A from precomputed digit chunks (bulk copies by thread 0 in cut; nothing to load)
template <int SA>
struct FillADigits {
    Smem& S;
    const uint16_t* digits;
    __device__ void load(int) {}
    __device__ void cut(int b, int c) { fill_A_digits<SA>(S, b, c, digits); }
};

// A from the rows of a row-major FP64 matrix X with row scales S.rowT: 128 rows x 4 groups of 8
// consecutive K, one group per thread
template <int SA>
struct FillARows {
    static_assert(L * (KC / 8) == kThreads, "one group per thread");
    Smem& S;
    const double* X;
    double2 v[4];
    __device__ void load(int c) {
        const int u = threadIdx.x;
        const int i = u & (L - 1), kg = u >> 7;
        const double* src = X + static_cast<size_t>(i) * L + c * KC + kg * 8;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = *reinterpret_cast<const double2*>(src + 2 * q);
    }
    __device__ void cut(int b, int c) {
        const int u = threadIdx.x;
        const int i = u & (L - 1), kg = u >> 7;
        const int T = S.rowT[i];
        unsigned long long U[8];
        bool neg[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            U[2 * q] = to_fixed_mag(v[q].x, T, neg[2 * q]);
            U[2 * q + 1] = to_fixed_mag(v[q].y, T, neg[2 * q + 1]);
        }
        store_digits<SA, 8>(U, neg, bufA(S, b, 0), A_SL, ((i >> 3) * 4 + kg) * 128 + (i & 7) * 16);
    }
};

// e_k = e^{V_k} as significand and exponent for sigma s_k = -1 (m0, E0) and +1 (m1, E1), passed
// as scalars and selected, never indexed, so that nothing of it goes to local memory.
struct EScale {
    unsigned long long m0, m1;
    int E0, E1;
};

// B from the columns p*NP .. p*NP+NP-1 of a row-major FP64 matrix X with column scales S.colT;
// with E, row k is multiplied by e_k (from es) exactly on the way.
// Each thread converts EPT = NP * KC / kThreads consecutive K of one column.
template <int SB, bool E, int NP>
struct FillBCols {
    static constexpr int EPT = NP * KC / kThreads;
    static_assert(EPT == 4 || EPT == 8, "4 or 8 K per thread");
    Smem& S;
    const double* X;
    int p;
    EScale es;
    double x[EPT];
    __device__ void load(int c) {
        const int t = threadIdx.x;
        const int jl = t & (NP - 1), k0 = (t / NP) * EPT;
        const int j = p * NP + jl;
#pragma unroll
        for (int q = 0; q < EPT; ++q) x[q] = X[static_cast<size_t>(c * KC + k0 + q) * L + j];
    }
    __device__ void cut(int b, int c) {
        const int t = threadIdx.x;
        const int jl = t & (NP - 1), k0 = (t / NP) * EPT;   // k0 within the chunk
        const int T = S.colT[p * NP + jl];
        unsigned long long U[EPT];
        bool neg[EPT];
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            if constexpr (E) {
                const bool up = S.s[c * KC + k0 + q] > 0;   // S.s holds sigma s_k
                U[q] = to_fixed_scaled_mag(x[q], up ? es.m1 : es.m0, up ? es.E1 : es.E0, T, neg[q]);
            } else {
                U[q] = to_fixed_mag(x[q], T, neg[q]);
            }
        }
        store_digits<SB, EPT>(U, neg, bufB<NP>(S, b, 0), NP * KC * 2,
                              ((jl >> 3) * 4 + (k0 >> 3)) * 128 + (jl & 7) * 16 + (k0 & 7) * 2);
    }
};

// ------------------------------------------------------------------------------------------
// one product pass: fills, MMAs, readout
// ------------------------------------------------------------------------------------------
// The MMAs of a chunk are issued by one thread.  Level n's accumulator is TMEM columns
// (n - 2) NP ...; for each digit s of A the digits t of B (whose chunk planes lie one after the
// other, NP rows each) are stacked along N in runs of at most 256 columns, one MMA per run and
// K half, writing the level blocks s + t ... in one go.  The first product of each level
// (s = max(1, n - SB), first chunk, first K half) overwrites its accumulator, and a run never
// mixes first products with later ones.  The schedules (first chunk, later chunks) are fixed at
// compile time.
struct ChunkRun {
    int kk, s, t, nt;
    bool first;
};
struct ChunkSchedule {
    ChunkRun run[64];
    int n;
};
template <int SA, int SB, int NL, int NP>
__host__ __device__ constexpr ChunkSchedule chunk_schedule(bool first_chunk) {
    constexpr int G = 256 / NP;
    ChunkSchedule S{};
    for (int kk = 0; kk < 2; ++kk)
        for (int s = 1; s <= SA; ++s) {
            const int tmax = SB < NL - s ? SB : NL - s;
            int t = 1;
            while (t <= tmax) {
                const auto first_of = [&](int tt) {
                    return first_chunk && kk == 0 && s == (s + tt - SB > 1 ? s + tt - SB : 1);
                };
                const bool first = first_of(t);
                int e = t;
                while (e < tmax && e - t + 1 < G && first_of(e + 1) == first) ++e;
                S.run[S.n++] = ChunkRun{kk, s, t, e - t + 1, first};
                t = e + 1;
            }
        }
    return S;
}

template <int SA, int SB, int NL, int NP, bool FIRST>
__device__ __forceinline__ void issue_runs(uint32_t tmem, uint64_t adesc, uint64_t bdesc) {
    constexpr ChunkSchedule S = chunk_schedule<SA, SB, NL, NP>(FIRST);
    static_assert(S.n <= 64, "schedule fits");
#pragma unroll
    for (int i = 0; i < S.n; ++i) {
        const ChunkRun r = S.run[i];
        mma_bf16(tmem + (r.s + r.t - 2) * NP, adesc + (((r.s - 1) * A_SL + r.kk * 256) >> 4),
                 bdesc + (((r.t - 1) * (NP * KC * 2) + r.kk * 256) >> 4), idesc_bf16_f32(128, r.nt * NP),
                 !r.first);
    }
}

template <int SA, int SB, int NL, int NP>
__device__ void issue_chunk(Smem& S, int b, int c) {
    tc_fence_after_sync();
    const uint64_t ad = smem_desc(smem_addr(bufA(S, b, 0)), 128, 512);
    const uint64_t bd = smem_desc(smem_addr(bufB<NP>(S, b, 0)), 128, 512);
    if (c == 0) issue_runs<SA, SB, NL, NP, true>(S.tmem, ad, bd);
    else issue_runs<SA, SB, NL, NP, false>(S.tmem, ad, bd);
    mma_commit(&S.mbar[b]);
}

// Runs one pass (output columns p*NP ...) of C = A B with the given operand fills (load / cut
// objects, see above) and hands every
// element's level sum Q (C_ij = Q 2^(rowT_i + colT_j - 54)) to the epilogue: pre(i, j0) once per
// 8 columns j0 ... j0+7 of row i (to load what the epilogue needs early), then epi(i, j, k, Q)
// for each, k = j - j0, which returns an exponent whose maximum over the rows lands in ncol[j]
// (when ncol is not null).  With TMA_A the A fill is a bulk copy whose completion the MMA issuer
// awaits.  Bit b of ph / tph tracks the phase of mbar[b] / tbar[b] (bit masks rather than
// arrays, so that the dynamic index b stays in registers).  Returns false if a wait ran out.
template <int SA, int SB, int NL, int NP, bool TMA_A, class FA, class FB, class PRE, class EPI>
__device__ bool product_pass(Smem& S, int p, uint32_t& ph, uint32_t& tph, FA& fillA,
                             FB& fillB, PRE pre, EPI epi, int* ncol) {
    static_assert(NL - 1 <= 8 && (NL - 1) * NP <= static_cast<int>(kTmemCols), "levels fit TMEM");
    static_assert(SB * NP * KC * 2 <= BUFB - SMAX * A_SL && SA <= SMAX, "digits fit the buffer");
    const int tid = threadIdx.x;
    bool ok = true;
    fillA.load(0);
    fillB.load(0);
    for (int c = 0; c < NCH; ++c) {
        const int b = c & 1;
        if (c >= 2) {   // the MMAs that read this buffer two chunks ago must be done
            ok = mbar_wait(&S.mbar[b], (ph >> b) & 1u) && ok;
            ph ^= 1u << b;
        }
        fillA.cut(b, c);
        fillB.cut(b, c);
        if (c + 1 < NCH) {
            fillA.load(c + 1);
            fillB.load(c + 1);
        }
        fence_async_shared();
        tc_fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            if constexpr (TMA_A) {
                ok = mbar_wait(&S.tbar[b], (tph >> b) & 1u) && ok;
            }
            issue_chunk<SA, SB, NL, NP>(S, b, c);
        }
        if constexpr (TMA_A) tph ^= 1u << b;
    }
    ok = mbar_wait(&S.mbar[0], ph & 1u) && ok;
    ok = mbar_wait(&S.mbar[1], (ph >> 1) & 1u) && ok;
    ph ^= 3u;
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after_sync();
    const int w = tid >> 5, lane = tid & 31;
    const int i = 32 * (w & 3) + lane;
    constexpr int NQ = kThreads / 128;   // warps per lane quarter
    const int cg = w >> 2;
    constexpr int G = NP / NQ / 8;       // groups of 8 columns per warp
    const uint32_t trow = S.tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16);
#pragma unroll 1
    for (int g = 0; g < G; ++g) {
        const int jl0 = (NP / NQ) * cg + 8 * g;
        pre(i, p * NP + jl0);
        long long Q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) Q[k] = 0;
        // the levels' columns in batches of up to four loads in flight per wait
#pragma unroll
        for (int n0 = 2; n0 <= NL; n0 += 4) {
            uint32_t r[4][8];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (n0 + u <= NL) tmem_ld8_async(trow + (n0 + u - 2) * NP + jl0, r[u]);
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (n0 + u <= NL) {
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        Q[k] += level_shift(static_cast<long long>(__float2int_rz(__uint_as_float(r[u][k]))), n0 + u);
                }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            // the epilogue returns its output's contribution to the next product's column
            // scale; the warp's 32 rows are folded by one redux, the four row blocks by atomics
            const int ce = epi(i, p * NP + jl0 + k, k, Q[k]);
            if (ncol) {
                const int m = __reduce_max_sync(0xffffffffu, ce);
                if (lane == 0) atomicMax(ncol + p * NP + jl0 + k, m);
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    return true;
}

// number of digit products (s, t) with s + t <= NL of two S-digit operands
__host__ __device__ constexpr int n_products(int S, int NL) {
    int n = 0;
    for (int s = 1; s <= S; ++s)
        for (int t = 1; t <= S; ++t)
            if (s + t <= NL) ++n;
    return n;
}

// ------------------------------------------------------------------------------------------
// operand scales
// ------------------------------------------------------------------------------------------
// colT[j] = max_k (exp(X_kj) + add_k) + 2 (+1 for the e scaling): |e_k X_kj| <= 2^(colT_j - 1)
__device__ void col_scales(Smem& S, const double* X, const int* Ee) {
    constexpr int NH = kThreads / L;   // threads per column
    const int t = threadIdx.x, j = t & (L - 1), h = t >> 7;
    int m = kNoExp;
    for (int k = h * (L / NH); k < (h + 1) * (L / NH); ++k) {
        int e = exp_of(X[static_cast<size_t>(k) * L + j]);
        if (Ee && e != kNoExp) e += Ee[S.s[k] > 0 ? 1 : 0] + 1;
        m = e > m ? e : m;
    }
    S.tmpT[t] = m;
    __syncthreads();
    if (t < L) {
        int a = S.tmpT[t];
        for (int q = 1; q < NH; ++q) a = max(a, S.tmpT[t + q * L]);
        S.colT[t] = a + 2;
    }
    __syncthreads();
}

// rowT[i] = max_k exp(X_ik) + 2, one warp per row at a time (coalesced)
__device__ void row_scales(Smem& S, const double* X) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = w; i < L; i += kThreads / 32) {
        int m = kNoExp;
#pragma unroll
        for (int q = 0; q < L / 32; ++q) {
            const int e = exp_of(X[static_cast<size_t>(i) * L + lane + 32 * q]);
            m = e > m ? e : m;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y > m ? y : m;
        }
        if (lane == 0) S.rowT[i] = m + 2;
    }
    __syncthreads();
}

// ------------------------------------------------------------------------------------------
// the refresh of one spin: X (FP32 state in Gf, FP64 iterate in Xa / Xb) -> G in Xa
// ------------------------------------------------------------------------------------------
struct SpinArgs {
    double* Xa;               // the chain's FP64 G of this spin (input: unused; output: G)
    double* Xb;               // scratch
    const float* Gf;          // FP32 state of this spin
    const uint16_t* digits;   // g0^{-1} digits of (site, spin)
    const int* rowTg;         // and its row scales
    EScale e;                 // e^V: significands and exponents for sigma s = -1 / +1
    EScale ev;                // |e^V - 1|
    bool evneg0, evneg1;      // e^V - 1 < 0 for sigma s = -1 / +1
};

// Moves the scales the last epilogue gathered into place: colT <- ncolT + 2 (and rowT <- nrowT +
// 2 with rows), and clears the gathering arrays.
__device__ void take_scales(Smem& S, bool rows) {
    __syncthreads();
    for (int i = threadIdx.x; i < L; i += kThreads) {
        S.colT[i] = S.ncolT[i] + 2;
        S.ncolT[i] = kNoExp;
        if (rows) {
            S.rowT[i] = S.nrowT[i] + 2;
            S.nrowT[i] = kNoExp;
        }
    }
    __syncthreads();
}

// R = 1 - g0^{-1} (E X) + D X for X in Xsrc (column scales of E X in S.colT), written to Rdst;
// returns max |R| (bit pattern key).  Gathers R's column scales and X's row scales for the
// correction that follows.
template <int S_, int NL>
__device__ bool residual(Smem& S, uint32_t& ph, uint32_t& tph, const SpinArgs& a,
                         const double* Xsrc, double* Rdst, unsigned long long& rmax) {
    constexpr int NP = 64;
    for (int i = threadIdx.x; i < L; i += kThreads) S.rowT[i] = S.gT[i];
    __syncthreads();
    if (threadIdx.x < 32) {   // largest row scale + largest column scale
        int mr = kNoExp, mc = kNoExp;
        for (int i = threadIdx.x; i < L; i += 32) {
            mr = S.rowT[i] > mr ? S.rowT[i] : mr;
            mc = S.colT[i] > mc ? S.colT[i] : mc;
        }
        mr = __reduce_max_sync(0xffffffffu, mr);
        mc = __reduce_max_sync(0xffffffffu, mc);
        if (threadIdx.x == 0 && mr + mc > kMaxScaleSum) S.flag = 1;
    }
    unsigned long long mx = 0;
    int xrow = kNoExp;   // this thread's row of X: largest exponent seen
    double xr[8];
    for (int p = 0; p < L / NP; ++p) {
        FillADigits<S_> fa{S, a.digits};
        FillBCols<S_, true, NP> fb{S, Xsrc, p, a.e};
        const bool ok = product_pass<S_, S_, NL, NP, true>(
            S, p, ph, tph, fa, fb,
            [&](int i, int j0) {
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                    const double2 v = *reinterpret_cast<const double2*>(Xsrc + static_cast<size_t>(i) * L + j0 + k);
                    xr[k] = v.x;
                    xr[k + 1] = v.y;
                }
            },
            [&](int i, int j, int k, long long Q) -> int {
                const int EQ = S.rowT[i] + S.colT[j] - 54;
                long long q = -Q;
                if (i == j) {
                    const int sh = -EQ;
                    if (sh < 0 || sh > 61) S.flag = 1;
                    else q += 1ll << sh;
                }
                const bool up = S.s[i] > 0;
                const int T = 62 + EQ;
                // |ev X| must lie below 2^(T - 1) for the fixed-point form; it does whenever the
                // scales are sane, otherwise the chain falls back
                const double x = xr[k];
                const int ex = exp_of(x);
                xrow = ex > xrow ? ex : xrow;
                const int Eev = up ? a.ev.E1 : a.ev.E0;
                if (ex != kNoExp && ex + Eev + 2 > T - 1) S.flag = 1;
                long long v = to_fixed_scaled(x, up ? a.ev.m1 : a.ev.m0, Eev, T);
                q += (up ? a.evneg1 : a.evneg0) ? -v : v;
                const double r = fixed_to_double(q, EQ);
                Rdst[static_cast<size_t>(i) * L + j] = r;
                const unsigned long long key =
                    static_cast<unsigned long long>(__double_as_longlong(r)) & 0x7FFFFFFFFFFFFFFFull;
                mx = key > mx ? key : mx;
                return exp_of(r);
            },
            S.ncolT);
        if (!ok) return false;
    }
    atomicMax(&S.nrowT[32 * ((threadIdx.x >> 5) & 3) + (threadIdx.x & 31)], xrow);
    rmax = block_max(S, mx);
    take_scales(S, true);   // rows: X's; columns: R's
    return true;
}

// X_new = X + X R (X in Xsrc with row scales S.rowT, R in Rsrc with column scales S.colT),
// written over Rsrc, in one pass of all 128 columns (4 digits, levels up to 5: the TMEM holds
// the four level accumulators of 128 columns).  Gathers the column scales of E X_new for the
// residual that follows.
template <int S_, int NL>
__device__ bool correct(Smem& S, uint32_t& ph, uint32_t& tph, const SpinArgs& a,
                        const double* Xsrc, double* Rsrc) {
    constexpr int NP = 128;
    double xr[8];
    FillARows<S_> fa{S, Xsrc};
    FillBCols<S_, false, NP> fb{S, Rsrc, 0, EScale{}};
    const bool ok = product_pass<S_, S_, NL, NP, false>(
        S, 0, ph, tph, fa, fb,
        [&](int i, int j0) {
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const double2 v = *reinterpret_cast<const double2*>(Xsrc + static_cast<size_t>(i) * L + j0 + k);
                xr[k] = v.x;
                xr[k + 1] = v.y;
            }
        },
        [&](int i, int j, int k, long long Q) -> int {
            const double x = xr[k] + fixed_to_double(Q, S.rowT[i] + S.colT[j] - 54);
            Rsrc[static_cast<size_t>(i) * L + j] = x;
            const int e = exp_of(x);
            return e == kNoExp ? kNoExp : e + (S.s[i] > 0 ? a.e.E1 : a.e.E0) + 1;
        },
        S.ncolT);
    if (!ok) return false;
    take_scales(S, false);  // columns: E X_new's
    return true;
}

__device__ bool refresh_spin(Smem& S, uint32_t& ph, uint32_t& tph, const SpinArgs& a,
                             int& products) {
    // X0 = the FP32 state, with the column scales of E X0; the row scales of g0^{-1}
    {
        constexpr int NH = kThreads / L, RH = L / NH;   // threads per column, rows per thread
        const int t = threadIdx.x, j = t & (L - 1), h = t >> 7;
        int m = kNoExp;
#pragma unroll 1
        for (int r0 = 0; r0 < RH; r0 += 16) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = a.Gf[static_cast<size_t>(h * RH + r0 + q) * L + j];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = h * RH + r0 + q;
                const double x = static_cast<double>(v[q]);
                a.Xa[static_cast<size_t>(k) * L + j] = x;
                const int e = exp_of(x);
                if (e != kNoExp) m = max(m, e + (S.s[k] > 0 ? a.e.E1 : a.e.E0) + 1);
            }
        }
        S.tmpT[t] = m;
        __syncthreads();
        if (t < L) {
            int mm = S.tmpT[t];
            for (int q = 1; q < NH; ++q) mm = max(mm, S.tmpT[t + q * L]);
            S.colT[t] = mm + 2;
            S.ncolT[t] = kNoExp;
            S.nrowT[t] = kNoExp;
            S.gT[t] = a.rowTg[t];
        }
        __syncthreads();
    }
    unsigned long long r = 0;
    // step 0: residual to about 2^-35 of the operand scales, enough that one full step then
    // converges from an FP32 state; correction from 4 digits (levels up to 5), which is what a
    // residual of that size needs
    if (!residual<7, 8>(S, ph, tph, a, a.Xa, a.Xb, r)) return false;
    products += n_products(7, 8);
    if (S.flag) return true;                                        // scales out of range
    if (exp_of(__longlong_as_double(static_cast<long long>(r))) >= kFarExp) {
        if (threadIdx.x == 0) S.flag = 1;                         // no approximate inverse
        __syncthreads();
        return true;
    }
    if (!correct<4, 5>(S, ph, tph, a, a.Xa, a.Xb)) return false;  // X1 in Xb
    products += n_products(4, 5);
    // full-accuracy steps until the residual is below 2^-24 (its square is then far below the
    // products' own error), at most two
    double* X = a.Xb;
    double* R = a.Xa;
    bool done = false;
    for (int it = 0; it < 2 && !done; ++it) {
        if (!residual<8, 9>(S, ph, tph, a, X, R, r)) return false;
        products += n_products(8, 9);
        if (S.flag) return true;
        if (!correct<4, 5>(S, ph, tph, a, X, R)) return false;    // X + X R over R
        products += n_products(4, 5);
        double* t = X;
        X = R;
        R = t;
        done = exp_of(__longlong_as_double(static_cast<long long>(r))) < kConvergedExp;
    }
    if (!done) {
        if (threadIdx.x == 0) S.flag = 1;
        __syncthreads();
        return true;
    }
    if (X != a.Xa) {   // the result belongs in the chain's G
        for (int e = threadIdx.x; e < LL; e += kThreads) a.Xa[e] = X[e];
        __syncthreads();
    }
    return true;
}

__device__ void split_e(double e, unsigned long long& m, int& E) { split_double(e, m, E); }

__global__ void __launch_bounds__(kThreads, 1)
refresh_tc_kernel(const QmcProblem P, const TcRefreshArgs A) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int c = blockIdx.x;
    if (c >= P.nchain) return;
    const int tid = threadIdx.x;
    const int site = c / P.cps;
    // after a timeout anywhere in this context, leave every chain to the Gauss-Jordan refresh
    if (*reinterpret_cast<volatile const int*>(P.status) == static_cast<int>(HF_ETIMEOUT)) {
        if (tid == 0) {
            A.fail[c] = 1;
            A.fail_list[atomicAdd(A.fail_count, 1)] = c;
        }
        return;
    }
    if (tid == 0) {
        S.flag = 0;
        S.timeout = 0;
        mbar_init(&S.mbar[0], 1);
        mbar_init(&S.mbar[1], 1);
        mbar_init(&S.tbar[0], 1);
        mbar_init(&S.tbar[1], 1);
        mbar_init_fence();
    }
    if (tid < 32) tmem_alloc(&S.tmem, kTmemCols);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    uint32_t ph = 0u, tph = 0u;
    const double e_p = 1.0 + P.ev_p, e_m = 1.0 + P.ev_m;
    bool ok = true;
    int products = 0;
    for (int sp = 0; sp < 2 && ok; ++sp) {
        const int sigma = sp == 0 ? 1 : -1;
        for (int l = tid; l < L; l += kThreads)
            S.s[l] = static_cast<int8_t>(sigma * P.s[static_cast<size_t>(c) * L + l]);
        SpinArgs a;
        a.Xa = P.G + (static_cast<size_t>(c) * 2 + sp) * LL;
        a.Xb = A.scratch + static_cast<size_t>(c) * LL;
        a.Gf = P.Gf + (static_cast<size_t>(c) * 2 + sp) * LL;
        a.digits = A.g0inv_digits + (static_cast<size_t>(site) * 2 + sp) * SMAX * LL;
        a.rowTg = A.g0inv_rowT + (static_cast<size_t>(site) * 2 + sp) * L;
        split_e(e_m, a.e.m0, a.e.E0);
        split_e(e_p, a.e.m1, a.e.E1);
        split_e(fabs(P.ev_m), a.ev.m0, a.ev.E0);
        split_e(fabs(P.ev_p), a.ev.m1, a.ev.E1);
        a.evneg0 = P.ev_m < 0.0;
        a.evneg1 = P.ev_p < 0.0;
        __syncthreads();
        ok = refresh_spin(S, ph, tph, a, products);
        if (!ok) {
            if (tid == 0) S.timeout = 1;
            break;
        }
        if (S.flag) break;
    }
    __syncthreads();
    tc_fence_after_sync();
    if (tid < 32) tmem_dealloc(S.tmem, kTmemCols);
    if (tid == 0 && A.products) atomicAdd(A.products, static_cast<unsigned long long>(products));
    if (S.timeout) {
        if (tid == 0) {
            atomicExch(P.status, static_cast<int>(HF_ETIMEOUT));
            A.fail[c] = 1;
            A.fail_list[atomicAdd(A.fail_count, 1)] = c;
        }
        return;
    }
    if (S.flag) {
        if (tid == 0) {
            A.fail[c] = 1;
            A.fail_list[atomicAdd(A.fail_count, 1)] = c;
            atomicAdd(reinterpret_cast<unsigned int*>(P.status + 7), 1u);
        }
        return;
    }
    if (tid == 0) {
        A.fail[c] = 0;
        atomicAdd(reinterpret_cast<unsigned int*>(P.status + 6), 1u);
    }
    // the FP32 copy (sweep state) and the drift of the state the sweeps reached
    float dv = 0.0f;
    const double* Gc = P.G + static_cast<size_t>(c) * 2 * LL;
    float* Gfc = P.Gf + static_cast<size_t>(c) * 2 * LL;
#pragma unroll 1
    for (int e0 = 0; e0 < 2 * LL; e0 += 8 * kThreads) {
        double x[8];
        float g[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            x[q] = Gc[e0 + q * kThreads + tid];
            g[q] = Gfc[e0 + q * kThreads + tid];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (P.drift) dv = fmaxf(dv, static_cast<float>(fabs(x[q] - static_cast<double>(g[q]))));
            Gfc[e0 + q * kThreads + tid] = static_cast<float>(x[q]);
        }
    }
    if (P.drift) drift_fold(P.drift, dv, tid == 0);
    if (P.refresh_measure) {
        __syncthreads();
        measure_refreshed<kThreads>(P, c, reinterpret_cast<double*>(S.tmpT));
    }
}

// digits and row scales of g0^{-1}, one CTA per (site, spin)
__global__ void __launch_bounds__(kThreads) g0inv_digits_kernel(const QmcProblem P, TcRefreshArgs A) {
    const int b = blockIdx.x;   // site * 2 + spin
    const double* G = P.g0inv + static_cast<size_t>(b) * LL;
    uint16_t* out = A.g0inv_digits + static_cast<size_t>(b) * SMAX * LL;
    int* rT = A.g0inv_rowT + static_cast<size_t>(b) * L;
    __shared__ int T[L];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = w; i < L; i += kThreads / 32) {
        int m = kNoExp;
        for (int q = 0; q < L / 32; ++q) {
            const int e = exp_of(G[static_cast<size_t>(i) * L + lane + 32 * q]);
            m = e > m ? e : m;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y > m ? y : m;
        }
        if (lane == 0) {
            T[i] = m + 2;
            rT[i] = m + 2;
        }
    }
    __syncthreads();
    // unit (i, kg): 8 consecutive K of row i; chunk c = kg / 4 holds its core column kg % 4
    for (int u = threadIdx.x; u < L * (L / 8); u += kThreads) {
        const int i = u & (L - 1), kg = u >> 7;
        const int c = kg >> 2, kgl = kg & 3;
        unsigned long long U[8];
        bool neg[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) U[q] = to_fixed_mag(G[static_cast<size_t>(i) * L + kg * 8 + q], T[i], neg[q]);
        unsigned char* base = reinterpret_cast<unsigned char*>(out) + static_cast<size_t>(c) * A_SL;
        store_digits<SMAX, 8>(U, neg, base, NCH * A_SL, ((i >> 3) * 4 + kgl) * 128 + (i & 7) * 16);
    }
}

// C = A B for independent 128 x 128 pairs (one CTA each), both operands with `SD` digits
template <int SD>
__global__ void __launch_bounds__(kThreads, 1)
tc_dgemm_kernel(const double* Am, const double* Bm, double* Cm, int n, int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const int m = blockIdx.x;
    if (m >= n) return;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&S.mbar[0], 1);
        mbar_init(&S.mbar[1], 1);
        mbar_init(&S.tbar[0], 1);
        mbar_init(&S.tbar[1], 1);
        mbar_init_fence();
    }
    if (tid < 32) tmem_alloc(&S.tmem, kTmemCols);
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    uint32_t ph = 0u, tph = 0u;
    const double* Ab = Am + static_cast<size_t>(m) * LL;
    const double* Bb = Bm + static_cast<size_t>(m) * LL;
    double* Cb = Cm + static_cast<size_t>(m) * LL;
    row_scales(S, Ab);
    col_scales(S, Bb, nullptr);
    bool ok = true;
    for (int p = 0; p < L / 64 && ok; ++p) {
        FillARows<SD> fa{S, Ab};
        FillBCols<SD, false, 64> fb{S, Bb, p, EScale{}};
        ok = product_pass<SD, SD, SD + 1, 64, false>(
            S, p, ph, tph, fa, fb,
            [&](int, int) {},
            [&](int i, int j, int, long long Q) -> int {
                Cb[static_cast<size_t>(i) * L + j] = fixed_to_double(Q, S.rowT[i] + S.colT[j] - 54);
                return kNoExp;
            },
            nullptr);
    }
    __syncthreads();
    tc_fence_after_sync();
    if (tid < 32) tmem_dealloc(S.tmem, kTmemCols);
    if (!ok && tid == 0 && status) atomicExch(status, static_cast<int>(HF_ETIMEOUT));
}

}  // namespace

size_t tc_digits_bytes(int nsite) { return static_cast<size_t>(nsite) * 2 * SMAX * LL * 2; }
size_t tc_refresh_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_g0inv_digits(const QmcProblem& p, const TcRefreshArgs& a, cudaStream_t st) {
    const int nb = 2 * (p.nchain / p.cps);
    if (nb <= 0) return cudaSuccess;
    g0inv_digits_kernel<<<nb, kThreads, 0, st>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_refresh_tc(const QmcProblem& p, const TcRefreshArgs& a, cudaStream_t st) {
    if (p.L != kTcL) return cudaErrorInvalidValue;
    const int smem = static_cast<int>(sizeof(Smem));
    cudaError_t e = cudaFuncSetAttribute(refresh_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (p.nchain <= 0) return cudaSuccess;
    refresh_tc_kernel<<<p.nchain, kThreads, smem, st>>>(p, a);
    return cudaGetLastError();
}

cudaError_t launch_tc_dgemm128(const double* A, const double* B, double* C, int n, int digits,
                               int* status, cudaStream_t st) {
    const int smem = static_cast<int>(sizeof(Smem));
    cudaError_t e = cudaSuccess;
    switch (digits) {
        case 1:
            e = cudaFuncSetAttribute(tc_dgemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess && n > 0) tc_dgemm_kernel<1><<<n, kThreads, smem, st>>>(A, B, C, n, status);
            break;
        case 3:
            e = cudaFuncSetAttribute(tc_dgemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess && n > 0) tc_dgemm_kernel<3><<<n, kThreads, smem, st>>>(A, B, C, n, status);
            break;
        case 5:
            e = cudaFuncSetAttribute(tc_dgemm_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess && n > 0) tc_dgemm_kernel<5><<<n, kThreads, smem, st>>>(A, B, C, n, status);
            break;
        case 7:
            e = cudaFuncSetAttribute(tc_dgemm_kernel<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess && n > 0) tc_dgemm_kernel<7><<<n, kThreads, smem, st>>>(A, B, C, n, status);
            break;
        case 8:
            e = cudaFuncSetAttribute(tc_dgemm_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e == cudaSuccess && n > 0) tc_dgemm_kernel<8><<<n, kThreads, smem, st>>>(A, B, C, n, status);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace hfk
