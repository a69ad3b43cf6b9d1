// k_qmc_f32.cu -- mixed-precision Hirsch-Fye QMC (sm_103a): FP32 sweeps, FP64 Dyson refresh.
//
// Sweeps (single-flip ratio, Metropolis test and Sherman-Morrison update of the Hirsch-Fye
// algorithm named in "Model and Methods") run in FP32 with FP32 accumulation, so that G_up and
// G_dn of a chain with L = 128 (2 x 64 KiB) stay in shared memory; accepted flips are applied as
// delayed rank-8 updates.  The refresh
// G = [1 + (1 - g0)(e^V - 1)]^{-1} g0 runs in FP64 in its own kernel, as the in-place
// Gauss-Jordan inversion of G^{-1} = g0^{-1} e^V - (e^V - 1) (L x L FP64, 128 KiB at L = 128,
// in shared memory), with g0^{-1} computed once per bath.  The refresh writes the FP64 G (used
// for the measurement that follows a refresh) and its FP32 copy (the sweep state).  One block
// of 256 threads per chain in both kernels.
#include <cuda_bf16.h>

#include <algorithm>

#include "hf_internal.cuh"
#include "k_refresh_tc.cuh"
#include "refresh_measure.cuh"
#include "tc_ozaki.cuh"

namespace hfk {
namespace {

constexpr int kT32 = 256;   // threads per block

// --------------------------------------------------------------------------------------------
// FP32 sweep kernel with delayed updates
//
// G_up and G_dn stay in shared memory (rows padded to L + 1 floats, so that a column read hits
// 32 different banks).  An accepted flip is not applied to G at once: its Sherman-Morrison factors
// u = (a / R)(G[:, l] - e_l) and w = G[l, :] (of the current G, pending updates included) are
// appended as column p of U and row p of W, and every kDK accepted flips (and at the end of the
// sweep) G += U W in one pass, kDK multiply-adds per element for one read and one write of it.
// The diagonal element a proposal needs, and the column and row an accepted flip needs, are G's
// plus the pending updates' contribution (O(kDK) per element).  The arithmetic is that of the
// rank-1 form reassociated, all in FP32 with FP32 accumulation.
// --------------------------------------------------------------------------------------------
constexpr int kDK = 8;   // pending rank-1 updates per spin

// L = 128: the flush G += U W runs on the tensor cores.  U and W^T are cut into three bf16 parts
// each (exact: 8 + 8 + 8 bits of an FP32 significand), the six part products with s + t <= 4 are
// accumulated in FP32 in TMEM (one 128 x 128 accumulator per spin; the dropped ones are below
// 2^-24 of |U||W|), and the sums are added to G in shared memory.  Operands: K-major core
// matrices, K = 16 (the 8 pending factors and 8 zeros).
constexpr int kTcFlushL = 128;
constexpr int kPartBytes = 128 * 16 * 2;   // one bf16 part of U or W^T: 128 rows x 16 K

__host__ __device__ constexpr size_t flush_tc_bytes(int L) {
    // parts[spin][U or W^T][3] + mbarrier + TMEM address
    return L == kTcFlushL ? static_cast<size_t>(2 * 2 * 3) * kPartBytes + 16 : 0;
}

__host__ __device__ constexpr size_t sweep32_bytes(int L) {
    // G[2][L][L+1] f32, U[2][L][kDK] f32, W[2][kDK][L] f32, u[L] f32 (even count), bacc[2L+3] f64,
    // red[32] f64, s[L] i8, then (L = 128) the tensor-core flush's operand parts
    return (static_cast<size_t>(2 * L * (L + 1) + 4 * L * kDK + L + (L & 1)) * 4 +
            static_cast<size_t>(2 * L + 3 + 32) * 8 + ((L + 15) / 16) * 16 + 16 + 1023) / 1024 * 1024 +
           flush_tc_bytes(L);
}

template <int L>
__device__ void measure32(const float* G0, const float* G1, double* bacc, double* red, int tid) {
    constexpr int LP = L + 1;
    for (int m = tid; m < L; m += kT32) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < L; ++q) {
            int l = q + m;
            if (l >= L) l -= L;
            int r = l + m;
            const bool wrap = r >= L;
            if (wrap) r -= L;
            const double x0 = G0[r * LP + l], x1 = G1[r * LP + l];
            s0 = wrap ? s0 - x0 : s0 + x0;
            s1 = wrap ? s1 - x1 : s1 + x1;
        }
        bacc[m] += s0 / L;
        bacc[L + m] += s1 / L;
    }
    double nu = 0.0, nd = 0.0, db = 0.0;
    for (int l = tid; l < L; l += kT32) {
        const double a = 1.0 - static_cast<double>(G0[l * LP + l]);
        const double b = 1.0 - static_cast<double>(G1[l * LP + l]);
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
    const int w = tid >> 5;
    if ((tid & 31) == 0) {
        red[w] = nu;
        red[8 + w] = nd;
        red[16 + w] = db;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int k = 0; k < kT32 / 32; ++k) {
            a += red[k];
            b += red[8 + k];
            c += red[16 + k];
        }
        bacc[2 * L + 0] += a / L;
        bacc[2 * L + 1] += b / L;
        bacc[2 * L + 2] += c / L;
    }
    __syncthreads();
}

// G += U W for the first m pending updates of both spins.  Thread t owns column t % L and rows
// t / L, t / L + kT32 / L, ...; W's column is kept in registers, each U row is read as two 16-byte
// broadcasts.
template <int L>
__device__ __forceinline__ void flush32(float* G0, float* G1, const float* U0, const float* U1,
                                        const float* W0, const float* W1, int m, int tid) {
    constexpr int LP = L + 1, STEP = kT32 / L;
    const int j = tid % L, i0 = tid / L;
    float w0[kDK], w1[kDK];
#pragma unroll
    for (int p = 0; p < kDK; ++p) {
        w0[p] = p < m ? W0[p * L + j] : 0.0f;
        w1[p] = p < m ? W1[p * L + j] : 0.0f;
    }
#pragma unroll 4
    for (int i = i0; i < L; i += STEP) {
        const float4 a0 = *reinterpret_cast<const float4*>(U0 + i * kDK);
        const float4 a1 = *reinterpret_cast<const float4*>(U0 + i * kDK + 4);
        const float4 b0 = *reinterpret_cast<const float4*>(U1 + i * kDK);
        const float4 b1 = *reinterpret_cast<const float4*>(U1 + i * kDK + 4);
        float g = G0[i * LP + j], h = G1[i * LP + j];
        g = fmaf(a0.x, w0[0], g);
        g = fmaf(a0.y, w0[1], g);
        g = fmaf(a0.z, w0[2], g);
        g = fmaf(a0.w, w0[3], g);
        g = fmaf(a1.x, w0[4], g);
        g = fmaf(a1.y, w0[5], g);
        g = fmaf(a1.z, w0[6], g);
        g = fmaf(a1.w, w0[7], g);
        h = fmaf(b0.x, w1[0], h);
        h = fmaf(b0.y, w1[1], h);
        h = fmaf(b0.z, w1[2], h);
        h = fmaf(b0.w, w1[3], h);
        h = fmaf(b1.x, w1[4], h);
        h = fmaf(b1.y, w1[5], h);
        h = fmaf(b1.z, w1[6], h);
        h = fmaf(b1.w, w1[7], h);
        G0[i * LP + j] = g;
        G1[i * LP + j] = h;
    }
}

struct FlushTc {
    unsigned char* parts;   // [spin][0: U, 1: W^T][3 parts] x kPartBytes, 1024-byte aligned
    uint64_t* bar;
    uint32_t* tmem;
};

// G_sigma += U_sigma W_sigma for the first m pending updates, on the tensor cores (L = 128).
// ph: the mbarrier's phase, flipped here.  Returns false if the wait ran out.
__device__ bool flush32_tc(float* G0, float* G1, const float* U0, const float* U1,
                           const float* W0, const float* W1, int m, int tid, const FlushTc& F,
                           uint32_t& ph) {
    constexpr int L = kTcFlushL, LP = L + 1;
    static_assert(kT32 == 2 * L, "one thread per (spin, row) of the operand parts");
    // three bf16 parts of each pending factor, zero beyond the m pending ones; thread t cuts
    // row t % 128 of U (t < 128: spin up) or of W^T (spin of t / 128 ... both spins each)
    {
        const int sp = tid >> 7, r = tid & 127;
        const float* U = sp ? U1 : U0;
        const float* W = sp ? W1 : W0;
        float uv[kDK], wv[kDK];
#pragma unroll
        for (int p = 0; p < kDK; ++p) {
            uv[p] = p < m ? U[r * kDK + p] : 0.0f;
            wv[p] = p < m ? W[p * L + r] : 0.0f;
        }
        unsigned char* Ub = F.parts + (sp * 2 + 0) * 3 * kPartBytes;
        unsigned char* Wb = F.parts + (sp * 2 + 1) * 3 * kPartBytes;
        const int off = (r >> 3) * 256 + (r & 7) * 16;   // core (r / 8, 0), row r % 8
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            float* v = side ? wv : uv;
            unsigned char* base = side ? Wb : Ub;
            uint32_t w[3][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float a0 = v[2 * q], a1 = v[2 * q + 1];
                uint32_t lo[3], hi[3];
#pragma unroll
                for (int pt = 0; pt < 3; ++pt) {
                    const __nv_bfloat16 b0 = __float2bfloat16_rn(a0), b1 = __float2bfloat16_rn(a1);
                    lo[pt] = __bfloat16_as_ushort(b0);
                    hi[pt] = __bfloat16_as_ushort(b1);
                    a0 -= __bfloat162float(b0);
                    a1 -= __bfloat162float(b1);
                }
#pragma unroll
                for (int pt = 0; pt < 3; ++pt) w[pt][q] = lo[pt] | (hi[pt] << 16);
            }
#pragma unroll
            for (int pt = 0; pt < 3; ++pt)
                *reinterpret_cast<uint4*>(base + pt * kPartBytes + off) =
                    make_uint4(w[pt][0], w[pt][1], w[pt][2], w[pt][3]);
        }
    }
    tc::fence_async_shared();
    tc::tc_fence_before_sync();
    __syncthreads();
    if (tid == 0) {
        tc::tc_fence_after_sync();
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128);
        constexpr int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            const uint32_t ua = tc::smem_addr(F.parts + (sp * 2 + 0) * 3 * kPartBytes);
            const uint32_t wa = tc::smem_addr(F.parts + (sp * 2 + 1) * 3 * kPartBytes);
#pragma unroll
            for (int k = 0; k < 6; ++k)
                tc::mma_bf16(*F.tmem + sp * 128, tc::smem_desc(ua + pa[k] * kPartBytes, 128, 256),
                             tc::smem_desc(wa + pb[k] * kPartBytes, 128, 256), idesc, k > 0);
        }
        tc::mma_commit(F.bar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait(F.bar, ph));
    ph ^= 1u;
    if (!ok) return false;
    tc::tc_fence_after_sync();
    {
        const int w = tid >> 5, lane = tid & 31;
        const int i = 32 * (w & 3) + lane, cg = w >> 2;
        const uint32_t trow = *F.tmem + (static_cast<uint32_t>(32 * (w & 3)) << 16);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            float* G = sp ? G1 : G0;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int j0 = 64 * cg + 16 * g;
                float v[16];
                tc::tmem_ld16(trow + sp * 128 + j0, v);
#pragma unroll
                for (int k = 0; k < 16; ++k) G[i * LP + j0 + k] += v[k];
            }
        }
    }
    tc::tc_fence_before_sync();
    return true;
}

template <int L>
__device__ void sweep32_chain(const QmcProblem& P, int c, unsigned char* base) {
    constexpr int LL = L * L;
    constexpr int LP = L + 1;
    constexpr int W = 2 * L + 3;
    static_assert(kT32 % L == 0 && L <= 128 && kDK == 8, "thread layout");
    const int tid = threadIdx.x;
    float* G0 = reinterpret_cast<float*>(base);
    float* G1 = G0 + L * LP;
    float* U0 = G1 + L * LP;                  // [L][kDK]
    float* U1 = U0 + L * kDK;
    float* W0 = U1 + L * kDK;                 // [kDK][L]
    float* W1 = W0 + kDK * L;
    float* u = W1 + kDK * L;
    double* bacc = reinterpret_cast<double*>(u + L + (L & 1));
    double* red = bacc + W;
    int8_t* s = reinterpret_cast<int8_t*>(red + 32);
    FlushTc ft{};
    uint32_t fph = 0u;
    bool tc_ok = true;
    if constexpr (L == kTcFlushL) {
        ft.parts = base + (sweep32_bytes(L) - flush_tc_bytes(L));
        ft.bar = reinterpret_cast<uint64_t*>(ft.parts + 2 * 2 * 3 * kPartBytes);
        ft.tmem = reinterpret_cast<uint32_t*>(ft.bar + 1);
        // the K padding (pending factors 8..15) stays zero: clear every part once
        for (int e = tid; e < 2 * 2 * 3 * kPartBytes / 16; e += kT32)
            reinterpret_cast<uint4*>(ft.parts)[e] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0) {
            tc::mbar_init(ft.bar, 1);
            tc::mbar_init_fence();
        }
        if (tid < 32) tc::tmem_alloc(ft.tmem, 256);
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
    }

    const int site = c / P.cps;
    const int ch = c - site * P.cps;
    const uint2 key = make_uint2(P.seed_lo, P.seed_hi);
    const float* Gg = P.Gf + static_cast<size_t>(c) * 2 * LL;
    for (int e = tid; e < LL; e += kT32) {
        const int i = e / L, j = e - (e / L) * L;
        G0[i * LP + j] = Gg[e];
        G1[i * LP + j] = Gg[LL + e];
    }
    for (int e = tid; e < 4 * L * kDK; e += kT32) U0[e] = 0.0f;   // U and W: no stale patterns
    for (int l = tid; l < L; l += kT32) s[l] = P.s[static_cast<size_t>(c) * L + l];
    uint32_t nsw = P.nsw[c];
    uint32_t nmeas = P.nmeas[c];
    unsigned long long acc = 0ull;
    double* bins_c = P.bins + static_cast<size_t>(c) * P.max_bins * W;
    int cur_bin = static_cast<int>(nmeas / P.bin_size);
    for (int k = tid; k < W; k += kT32)
        bacc[k] = (cur_bin < P.max_bins) ? bins_c[static_cast<size_t>(cur_bin) * W + k] : 0.0;
    __syncthreads();

    for (int k = 0; k < P.nsweeps; ++k) {
        for (int l = tid; l < L; l += kT32)
            u[l] = uniform24(philox4x32_10(make_uint4(nsw, static_cast<uint32_t>(l),
                                                      static_cast<uint32_t>(ch),
                                                      static_cast<uint32_t>(P.site0 + site)), key));
        __syncthreads();
        int m = 0;   // pending updates (block-uniform)
        for (int l = 0; l < L; ++l) {
            // the current diagonal: G_ll plus the pending updates' part
            float g0 = G0[l * LP + l], g1 = G1[l * LP + l];
            for (int p = 0; p < m; ++p) {
                g0 = fmaf(U0[l * kDK + p], W0[p * L + l], g0);
                g1 = fmaf(U1[l * kDK + p], W1[p * L + l], g1);
            }
            const int sl = s[l];
            const float au = (sl > 0) ? P.af_p : P.af_m;
            const float ad = (sl > 0) ? P.af_m : P.af_p;
            const float Ru = 1.0f + (1.0f - g0) * au;
            const float Rd = 1.0f + (1.0f - g1) * ad;
            const float pr = Ru * Rd;
            if (!(pr > 0.0f) && tid == 0) atomicAdd(P.status + 1, 1);
            if (u[l] < pr) {
                const float fu = au / Ru, fd = ad / Rd;
                if (tid < L) {                     // column l of the current G -> U[:, m]
                    const int i = tid;
                    float c0 = G0[i * LP + l], c1 = G1[i * LP + l];
                    for (int p = 0; p < m; ++p) {
                        c0 = fmaf(U0[i * kDK + p], W0[p * L + l], c0);
                        c1 = fmaf(U1[i * kDK + p], W1[p * L + l], c1);
                    }
                    const float one = (i == l) ? 1.0f : 0.0f;
                    U0[i * kDK + m] = fu * (c0 - one);
                    U1[i * kDK + m] = fd * (c1 - one);
                } else if (tid >= 128 && tid < 128 + L) {   // row l -> W[m, :]
                    const int j = tid - 128;
                    float r0 = G0[l * LP + j], r1 = G1[l * LP + j];
                    for (int p = 0; p < m; ++p) {
                        r0 = fmaf(U0[l * kDK + p], W0[p * L + j], r0);
                        r1 = fmaf(U1[l * kDK + p], W1[p * L + j], r1);
                    }
                    W0[m * L + j] = r0;
                    W1[m * L + j] = r1;
                }
                __syncthreads();
                if (tid == 0) s[l] = static_cast<int8_t>(-sl);
                ++acc;
                if (++m == kDK) {
                    if constexpr (L == kTcFlushL) tc_ok = tc_ok && flush32_tc(G0, G1, U0, U1, W0, W1, m, tid, ft, fph);
                    else flush32<L>(G0, G1, U0, U1, W0, W1, m, tid);
                    m = 0;
                    __syncthreads();
                }
            }
        }
        if (m > 0) {
            if constexpr (L == kTcFlushL) tc_ok = tc_ok && flush32_tc(G0, G1, U0, U1, W0, W1, m, tid, ft, fph);
            else flush32<L>(G0, G1, U0, U1, W0, W1, m, tid);
        }
        ++nsw;
        __syncthreads();
        if (k >= P.meas_from && k < P.meas_to) {
            measure32<L>(G0, G1, bacc, red, tid);
            ++nmeas;
            if (nmeas % static_cast<uint32_t>(P.bin_size) == 0u) {
                const int b = static_cast<int>(nmeas / P.bin_size) - 1;
                for (int q = tid; q < W; q += kT32) {
                    if (b < P.max_bins) bins_c[static_cast<size_t>(b) * W + q] = bacc[q];
                    bacc[q] = 0.0;
                }
                __syncthreads();
            }
        }
    }
    cur_bin = static_cast<int>(nmeas / P.bin_size);
    for (int q = tid; q < W; q += kT32)
        if (cur_bin < P.max_bins) bins_c[static_cast<size_t>(cur_bin) * W + q] = bacc[q];
    float* Gw = P.Gf + static_cast<size_t>(c) * 2 * LL;
    for (int e = tid; e < LL; e += kT32) {
        const int i = e / L, j = e - (e / L) * L;
        Gw[e] = G0[i * LP + j];
        Gw[LL + e] = G1[i * LP + j];
    }
    for (int l = tid; l < L; l += kT32) P.s[static_cast<size_t>(c) * L + l] = s[l];
    if (tid == 0) {
        P.nsw[c] = nsw;
        P.nmeas[c] = nmeas;
        P.acc[c] += acc;
    }
    if constexpr (L == kTcFlushL) {
        __syncthreads();
        tc::tc_fence_after_sync();
        if (tid < 32) tc::tmem_dealloc(*ft.tmem, 256);
        if (!tc_ok && tid == 0) atomicExch(P.status, static_cast<int>(HF_ETIMEOUT));
    }
}

__global__ void __launch_bounds__(kT32) qmc_f32_kernel(const __grid_constant__ QmcBatch B) {
    extern __shared__ __align__(1024) unsigned char smem[];
    int pi = 0;
    while (pi + 1 < B.nprob && static_cast<int>(blockIdx.x) >= B.p[pi + 1].block0) ++pi;
    const QmcProblem& P = B.p[pi];
    const int c = static_cast<int>(blockIdx.x) - P.block0;
    if (c >= P.nchain) return;
    switch (P.L) {
        case 16: sweep32_chain<16>(P, c, smem); break;
        case 32: sweep32_chain<32>(P, c, smem); break;
        case 64: sweep32_chain<64>(P, c, smem); break;
        case 128: sweep32_chain<128>(P, c, smem); break;
        default: break;
    }
}

// --------------------------------------------------------------------------------------------
// FP64 refresh (one block per chain, both spins) by way of the inverse Green function.
// A G = g0 with A = 1 + (1 - g0) D, D = diag(e^V - 1), gives G^{-1} = g0^{-1} A =
// g0^{-1} e^V - D.  With g0^{-1} computed once per bath (launch_g0_inverse), a refresh is one
// in-place Gauss-Jordan inversion of M = g0^{-1} e^V - D: L^3 FP64 multiply-adds, against the
// (4/3) L^3 of factoring A and solving for the L columns of g0, and every elimination step is a
// full-width rank-1 update that all threads share evenly.
// --------------------------------------------------------------------------------------------
__host__ __device__ constexpr size_t refresh_bytes(int L) {
    // M[L*L] f64, fcol[L] f64, red[32] f64, scal[2] f64, piv[L] int, flag[4] int
    return static_cast<size_t>(L * L + L + 32 + 2) * 8 + static_cast<size_t>(L + 4) * 4;
}

__device__ __forceinline__ unsigned long long mag64(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

struct GjScratch {
    double* M;      // [L][L] the matrix, inverted in place
    double* fcol;   // [L] the pivot column of the current step
    double* red;    // [32] reduction scratch
    double* scal;   // [2] reciprocal of the pivot
    int* piv;       // [L] pivot row of each step
    int* flag;      // [4] pivot row, zero-pivot flag
};

template <int L>
__device__ GjScratch gj_scratch(unsigned char* smem) {
    GjScratch g;
    g.M = reinterpret_cast<double*>(smem);
    g.fcol = g.M + L * L;
    g.red = g.fcol + L;
    g.scal = g.red + 32;
    g.piv = reinterpret_cast<int*>(g.scal + 2);
    g.flag = g.piv + L;
    return g;
}

// In-place Gauss-Jordan inversion of the row-major L x L matrix g.M with partial pivoting by
// rows, by kT32 threads: each step takes the largest |M[i][k]|, i >= k, as pivot, swaps it into
// row k, scales row k by its reciprocal, moves column k out and subtracts its multiples of row
// k from every other row; the column order is restored at the end.  Each thread owns column
// tid % L and rows tid / L + n (kT32 / L); its rows go in register groups of up to 8 (all
// loads, then the multiply-adds, then the stores).  Returns false if a pivot column was zero.
template <int L>
__device__ bool gj_invert(const GjScratch& g, int tid) {
    constexpr int STEP = kT32 / L, NR = L / STEP, GB = NR < 8 ? NR : 8;
    static_assert(kT32 % L == 0 && NR * STEP == L && NR % GB == 0, "thread layout");
    double* M = g.M;
    const int j = tid % L, i0 = tid / L;
    bool ok = true;
    for (int k = 0; k < L; ++k) {
        if (tid < 32) {
            unsigned long long best = 0ull;
            int bi = L;
            for (int i = k + tid; i < L; i += 32) {
                const unsigned long long key = mag64(M[i * L + k]);
                if (bi == L || key > best) {
                    best = key;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (oi != L && (bi == L || ob > best || (ob == best && oi < bi))) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) {
                g.piv[k] = bi;
                g.flag[0] = bi;
                g.flag[1] = (best == 0ull) ? 1 : 0;
                g.scal[0] = 1.0 / M[bi * L + k];
            }
        }
        __syncthreads();
        const int p = g.flag[0];
        if (g.flag[1]) ok = false;
        if (p != k) {
            for (int jj = tid; jj < L; jj += kT32) {
                const double t = M[k * L + jj];
                M[k * L + jj] = M[p * L + jj];
                M[p * L + jj] = t;
            }
            __syncthreads();
        }
        const double pinv = g.scal[0];
        // disjoint elements: row k (scaled; its diagonal becomes the reciprocal) and the rest of
        // column k (copied out and zeroed)
        for (int jj = tid; jj < L; jj += kT32) {
            const double x = M[k * L + jj];
            M[k * L + jj] = (jj == k) ? pinv : x * pinv;
        }
        for (int i = tid; i < L; i += kT32) {
            if (i != k) {
                g.fcol[i] = M[i * L + k];
                M[i * L + k] = 0.0;
            } else {
                g.fcol[i] = 0.0;   // row k subtracts nothing from itself
            }
        }
        __syncthreads();
        const double rk = M[k * L + j];
        for (int b = 0; b < NR; b += GB) {
            double a[GB], f[GB];
#pragma unroll
            for (int q = 0; q < GB; ++q) {
                const int i = i0 + (b + q) * STEP;
                a[q] = M[i * L + j];
                f[q] = g.fcol[i];
            }
#pragma unroll
            for (int q = 0; q < GB; ++q) a[q] = fma(-f[q], rk, a[q]);
#pragma unroll
            for (int q = 0; q < GB; ++q) {
                const int i = i0 + (b + q) * STEP;
                if (i != k) M[i * L + j] = a[q];
            }
        }
        __syncthreads();
    }
    for (int k = L - 1; k >= 0; --k) {   // undo the row swaps as column swaps, last first
        const int p = g.piv[k];
        if (p != k) {
            for (int i = tid; i < L; i += kT32) {
                const double t = M[i * L + k];
                M[i * L + k] = M[i * L + p];
                M[i * L + p] = t;
            }
            __syncthreads();
        }
    }
    return ok;
}

// G_sigma = M^{-1}, M = g0^{-1} e^{V_sigma} - (e^{V_sigma} - 1) (columns scaled by the fields)
template <int L>
__device__ bool refresh_chain(const QmcProblem& P, int c, unsigned char* smem) {
    const int tid = threadIdx.x;
    const GjScratch g = gj_scratch<L>(smem);
    constexpr int LL = L * L;
    const int site = c / P.cps;
    const int8_t* s = P.s + static_cast<size_t>(c) * L;
    double* Gout = P.G + static_cast<size_t>(c) * 2 * LL;
    float* Gf = P.Gf ? P.Gf + static_cast<size_t>(c) * 2 * LL : nullptr;
    const double ex_p = 1.0 + P.ev_p, ex_m = 1.0 + P.ev_m;
    bool ok = true;
    float dv = 0.0f;
    for (int sp = 0; sp < 2; ++sp) {
        const int sigma = sp == 0 ? 1 : -1;
        const double* gi = P.g0inv + (static_cast<size_t>(site) * 2 + sp) * LL;
        for (int e = tid; e < LL; e += kT32) {
            const int i = e / L, j = e - (e / L) * L;
            const bool up = sigma * s[j] > 0;
            const double m = gi[e] * (up ? ex_p : ex_m);
            g.M[e] = (i == j) ? m - (up ? P.ev_p : P.ev_m) : m;
        }
        __syncthreads();
        ok = gj_invert<L>(g, tid) && ok;
        for (int e = tid; e < LL; e += kT32) {
            const double x = g.M[e];
            Gout[static_cast<size_t>(sp) * LL + e] = x;
            if (Gf) {
                // drift monitor: the FP32 state the sweeps reached against the Dyson solution
                if (P.drift) dv = fmaxf(dv, static_cast<float>(fabs(x - Gf[static_cast<size_t>(sp) * LL + e])));
                Gf[static_cast<size_t>(sp) * LL + e] = static_cast<float>(x);
            }
        }
        __syncthreads();
    }
    if (P.drift) drift_fold(P.drift, dv, tid == 0);
    return ok;
}

// Refresh (and, with refresh_measure, measure) chain c.
__device__ void refresh_one(const QmcProblem& P, int c, unsigned char* smem) {
    const int L = P.L;
    const int tid = threadIdx.x;
    const int LL = L * L;
    bool ok = true;
    switch (L) {
        case 16: ok = refresh_chain<16>(P, c, smem); break;
        case 32: ok = refresh_chain<32>(P, c, smem); break;
        case 64: ok = refresh_chain<64>(P, c, smem); break;
        case 128: ok = refresh_chain<128>(P, c, smem); break;
        default: break;
    }
    double* red = reinterpret_cast<double*>(smem) + LL + L;
    if (!ok && tid == 0) atomicExch(P.status, static_cast<int>(HF_ENUMERIC));
    if (!P.refresh_measure) return;
    // measurement from the FP64 G just written (this block wrote it; block-wide visibility)
    __threadfence_block();
    __syncthreads();
    measure_refreshed<kT32>(P, c, red);
}

// every chain (list == nullptr: one CTA per chain) or the listed ones (a wave of CTAs that take
// list[k], k = blockIdx.x, blockIdx.x + gridDim.x, ... < *count)
__global__ void __launch_bounds__(kT32, 1) refresh_f64_kernel(const QmcProblem P, const int* list,
                                                           const int* count) {
    extern __shared__ __align__(1024) unsigned char smem[];
    if (!list) {
        if (static_cast<int>(blockIdx.x) < P.nchain) refresh_one(P, blockIdx.x, smem);
        return;
    }
    const int n = *count;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        refresh_one(P, list[k], smem);
        __syncthreads();   // the next chain reuses the shared memory
    }
}

}  // namespace

bool qmc_f32_supported(int L) { return L == 16 || L == 32 || L == 64 || L == 128; }
int qmc_f32_chains_per_block(int) { return 1; }
size_t qmc_f32_smem_bytes(int L) { return sweep32_bytes(L); }
size_t refresh_f64_smem_bytes(int L) { return refresh_bytes(L); }

cudaError_t launch_qmc_f32(const QmcBatch& b, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(qmc_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(sweep32_bytes(128)));
    if (e != cudaSuccess) return e;
    if (b.nblocks <= 0) return cudaSuccess;
    qmc_f32_kernel<<<b.nblocks, kT32, smem, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_refresh_f64(const QmcProblem& p, cudaStream_t st) {
    const size_t smem = refresh_bytes(p.L);
    cudaError_t e = cudaFuncSetAttribute(refresh_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(refresh_bytes(128)));
    if (e != cudaSuccess) return e;
    if (p.nchain <= 0) return cudaSuccess;
    refresh_f64_kernel<<<p.nchain, kT32, smem, st>>>(p, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_refresh_f64_listed(const QmcProblem& p, const int* list, const int* count,
                                      cudaStream_t st) {
    const size_t smem = refresh_bytes(p.L);
    cudaError_t e = cudaFuncSetAttribute(refresh_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(refresh_bytes(128)));
    if (e != cudaSuccess) return e;
    if (p.nchain <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    refresh_f64_kernel<<<std::min(p.nchain, sms), kT32, smem, st>>>(p, list, count);
    return cudaGetLastError();
}

}  // namespace hfk
