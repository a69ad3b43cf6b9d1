// k_qmc_f32.cu -- mixed-precision Hirsch-Fye QMC (sm_103a): FP32 sweeps, FP64 Dyson refresh.
//
// Sweeps (single-flip ratio, Metropolis test, Sherman-Morrison update of "Model and Methods"
// with the ratio of the benchmark spec) run in FP32 with FP32 accumulation, so that G_up and G_dn of
// a chain with L = 128 (2 x 64 KiB) stay in shared memory.  The refresh
// G = [1 + (1 - g0)(e^V - 1)]^{-1} g0 runs in FP64 in its own kernel: A (L x L FP64, 128 KiB at
// L = 128) is LU-factored with partial pivoting in shared memory and the right-hand side g0
// (rebuilt from g~0(tau) on the fly) is solved in blocks of 32 columns.  The refresh writes the
// FP64 G (used for the measurement that follows a refresh) and its FP32 copy (the sweep state).
// One block of 256 threads per chain in both kernels.
#include <algorithm>

#include "hf_internal.cuh"

namespace hfk {
namespace {

constexpr int kT32 = 256;   // threads per block
constexpr int kRhsBlock = 32;

// --------------------------------------------------------------------------------------------
// FP32 sweep kernel
// --------------------------------------------------------------------------------------------
__host__ __device__ constexpr size_t sweep32_bytes(int L) {
    // Gf[2][L*L] f32, cr[4L] f32, u[L] f32, bacc[2L+3] f64, red[32] f64, s[L] i8
    return static_cast<size_t>(2 * L * L + 5 * L) * 4 + static_cast<size_t>(2 * L + 3 + 32) * 8 +
           ((L + 15) / 16) * 16 + 16;
}

template <int L>
__device__ void measure32(const float* G0, const float* G1, double* bacc, double* red, int tid) {
    for (int m = tid; m < L; m += kT32) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < L; ++q) {
            int l = q + m;
            if (l >= L) l -= L;
            int r = l + m;
            const bool wrap = r >= L;
            if (wrap) r -= L;
            const double x0 = G0[r * L + l], x1 = G1[r * L + l];
            s0 = wrap ? s0 - x0 : s0 + x0;
            s1 = wrap ? s1 - x1 : s1 + x1;
        }
        bacc[m] += s0 / L;
        bacc[L + m] += s1 / L;
    }
    double nu = 0.0, nd = 0.0, db = 0.0;
    for (int l = tid; l < L; l += kT32) {
        const double a = 1.0 - static_cast<double>(G0[l * L + l]);
        const double b = 1.0 - static_cast<double>(G1[l * L + l]);
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

template <int L>
__device__ void sweep32_chain(const QmcProblem& P, int c, unsigned char* base) {
    constexpr int LL = L * L;
    constexpr int W = 2 * L + 3;
    static_assert(kT32 % L == 0, "one column per thread");
    const int tid = threadIdx.x;
    float* G0 = reinterpret_cast<float*>(base);
    float* G1 = G0 + LL;
    float* cr = G1 + LL;
    float* u = cr + 4 * L;
    double* bacc = reinterpret_cast<double*>(u + L + ((L & 1) ? 1 : 0));
    double* red = bacc + W;
    int8_t* s = reinterpret_cast<int8_t*>(red + 32);

    const int site = c / P.cps;
    const int ch = c - site * P.cps;
    const uint2 key = make_uint2(P.seed_lo, P.seed_hi);
    const float* Gg = P.Gf + static_cast<size_t>(c) * 2 * LL;
    for (int e = tid; e < LL; e += kT32) {
        G0[e] = Gg[e];
        G1[e] = Gg[LL + e];
    }
    for (int l = tid; l < L; l += kT32) s[l] = P.s[static_cast<size_t>(c) * L + l];
    uint32_t nsw = P.nsw[c];
    uint32_t nmeas = P.nmeas[c];
    unsigned long long acc = 0ull;
    double* bins_c = P.bins + static_cast<size_t>(c) * P.max_bins * W;
    int cur_bin = static_cast<int>(nmeas / P.bin_size);
    for (int k = tid; k < W; k += kT32)
        bacc[k] = (cur_bin < P.max_bins) ? bins_c[static_cast<size_t>(cur_bin) * W + k] : 0.0;
    __syncthreads();

    const int j = tid % L;
    const int i0 = tid / L;
    for (int k = 0; k < P.nsweeps; ++k) {
        for (int l = tid; l < L; l += kT32)
            u[l] = uniform24(philox4x32_10(make_uint4(nsw, static_cast<uint32_t>(l),
                                                      static_cast<uint32_t>(ch),
                                                      static_cast<uint32_t>(P.site0 + site)), key));
        __syncthreads();
        for (int l = 0; l < L; ++l) {
            const float g0 = G0[l * L + l], g1 = G1[l * L + l];
            const int sl = s[l];
            const float au = (sl > 0) ? P.af_p : P.af_m;
            const float ad = (sl > 0) ? P.af_m : P.af_p;
            const float Ru = 1.0f + (1.0f - g0) * au;
            const float Rd = 1.0f + (1.0f - g1) * ad;
            const float p = Ru * Rd;
            if (!(p > 0.0f) && tid == 0) atomicAdd(P.status + 1, 1);
            if (u[l] < p) {
                const float fu = au / Ru, fd = ad / Rd;
                for (int i = tid; i < L; i += kT32) {
                    const float one = (i == l) ? 1.0f : 0.0f;
                    cr[i] = fu * (G0[i * L + l] - one);
                    cr[L + i] = fd * (G1[i * L + l] - one);
                    cr[2 * L + i] = G0[l * L + i];
                    cr[3 * L + i] = G1[l * L + i];
                }
                __syncthreads();
                const float r0 = cr[2 * L + j], r1 = cr[3 * L + j];
#pragma unroll 8
                for (int i = i0; i < L; i += kT32 / L) {
                    G0[i * L + j] = fmaf(cr[i], r0, G0[i * L + j]);
                    G1[i * L + j] = fmaf(cr[L + i], r1, G1[i * L + j]);
                }
                __syncthreads();
                if (tid == 0) s[l] = static_cast<int8_t>(-sl);
                ++acc;
            }
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
        Gw[e] = G0[e];
        Gw[LL + e] = G1[e];
    }
    for (int l = tid; l < L; l += kT32) P.s[static_cast<size_t>(c) * L + l] = s[l];
    if (tid == 0) {
        P.nsw[c] = nsw;
        P.nmeas[c] = nmeas;
        P.acc[c] += acc;
    }
}

__global__ void __launch_bounds__(kT32) qmc_f32_kernel(const __grid_constant__ QmcBatch B) {
    extern __shared__ __align__(16) unsigned char smem[];
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
// FP64 refresh kernel (one block per chain, both spins)
// --------------------------------------------------------------------------------------------
__host__ __device__ constexpr size_t refresh_bytes(int L) {
    // A[L*L] f64, B[L*32] f64, f[L] f64, red[32] f64, perm[L] int, flag[4] int
    return static_cast<size_t>(L * L + L * kRhsBlock + L + 32) * 8 + static_cast<size_t>(L + 4) * 4;
}

__device__ __forceinline__ unsigned long long mag64(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

__global__ void __launch_bounds__(kT32) refresh_f64_kernel(const QmcProblem P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = P.L;
    const int c = blockIdx.x;
    if (c >= P.nchain) return;
    const int tid = threadIdx.x;
    double* A = reinterpret_cast<double*>(smem);
    double* B = A + L * L;
    double* f = B + L * kRhsBlock;
    double* red = f + L;
    int* perm = reinterpret_cast<int*>(red + 32);
    int* flag = perm + L;
    const int site = c / P.cps;
    const int LL = L * L;
    const int8_t* s = P.s + static_cast<size_t>(c) * L;
    double* Gout = P.G + static_cast<size_t>(c) * 2 * LL;
    float* Gf = P.Gf ? P.Gf + static_cast<size_t>(c) * 2 * LL : nullptr;
    bool ok = true;
    for (int sp = 0; sp < 2; ++sp) {
        const int sigma = sp == 0 ? 1 : -1;
        const double* gt = P.gtau + (static_cast<size_t>(site) * 2 + sp) * L;
        // A = 1 + (1 - g0) diag(e^{lambda sigma s_j} - 1)
        for (int e = tid; e < LL; e += kT32) {
            const int i = e / L, j = e - (e / L) * L;
            const int d = i - j;
            const double g = (d >= 0) ? gt[d] : -gt[d + L];
            const double ev = (sigma * s[j] > 0) ? P.ev_p : P.ev_m;
            const double one = (i == j) ? 1.0 : 0.0;
            A[e] = __dadd_rn(one, __dmul_rn(__dadd_rn(one, -g), ev));
        }
        for (int i = tid; i < L; i += kT32) perm[i] = i;
        __syncthreads();
        // LU with partial pivoting, in place (unit-lower multipliers below the diagonal)
        for (int k = 0; k < L; ++k) {
            if (tid < 32) {
                unsigned long long best = 0ull;
                int bi = L;
                for (int i = k + tid; i < L; i += 32) {
                    const unsigned long long key = mag64(A[i * L + k]);
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
                    flag[0] = bi;
                    flag[1] = (best == 0ull) ? 1 : 0;
                    if (bi != k) {
                        const int t = perm[k];
                        perm[k] = perm[bi];
                        perm[bi] = t;
                    }
                }
            }
            __syncthreads();
            const int p = flag[0];
            if (flag[1]) ok = false;
            if (p != k)
                for (int jj = tid; jj < L; jj += kT32) {
                    const double t = A[k * L + jj];
                    A[k * L + jj] = A[p * L + jj];
                    A[p * L + jj] = t;
                }
            __syncthreads();
            const double inv = 1.0 / A[k * L + k];
            for (int i = k + 1 + tid; i < L; i += kT32) {
                const double m = A[i * L + k] * inv;
                f[i] = m;
                A[i * L + k] = m;
            }
            __syncthreads();
            const int rows = L - 1 - k, cols = L - 1 - k;
            for (int e = tid; e < rows * cols; e += kT32) {
                const int r = e / cols;
                const int i = k + 1 + r, jj = k + 1 + (e - r * cols);
                A[i * L + jj] = fma(-f[i], A[k * L + jj], A[i * L + jj]);
            }
            __syncthreads();
        }
        // solve for g0 in blocks of 32 columns: X = U^{-1} L^{-1} P g0
        for (int c0 = 0; c0 < L; c0 += kRhsBlock) {
            const int nc = min(kRhsBlock, L - c0);
            for (int e = tid; e < L * nc; e += kT32) {
                const int i = e / nc, cc = e - (e / nc) * nc;
                const int r = perm[i], col = c0 + cc;
                const int d = r - col;
                B[i * kRhsBlock + cc] = (d >= 0) ? gt[d] : -gt[d + L];
            }
            __syncthreads();
            for (int k = 0; k < L; ++k) {        // forward, unit lower
                for (int e = tid; e < (L - 1 - k) * nc; e += kT32) {
                    const int r = e / nc, cc = e - r * nc;
                    const int i = k + 1 + r;
                    B[i * kRhsBlock + cc] = fma(-A[i * L + k], B[k * kRhsBlock + cc], B[i * kRhsBlock + cc]);
                }
                __syncthreads();
            }
            for (int k = L - 1; k >= 0; --k) {   // backward, upper
                if (tid < nc) B[k * kRhsBlock + tid] = B[k * kRhsBlock + tid] / A[k * L + k];
                __syncthreads();
                for (int e = tid; e < k * nc; e += kT32) {
                    const int i = e / nc, cc = e - (e / nc) * nc;
                    B[i * kRhsBlock + cc] = fma(-A[i * L + k], B[k * kRhsBlock + cc], B[i * kRhsBlock + cc]);
                }
                __syncthreads();
            }
            for (int e = tid; e < L * nc; e += kT32) {
                const int i = e / nc, cc = e - (e / nc) * nc;
                const double x = B[i * kRhsBlock + cc];
                Gout[static_cast<size_t>(sp) * LL + i * L + c0 + cc] = x;
                if (Gf) Gf[static_cast<size_t>(sp) * LL + i * L + c0 + cc] = static_cast<float>(x);
            }
            __syncthreads();
        }
    }
    if (!ok && tid == 0) atomicExch(P.status, static_cast<int>(HF_ENUMERIC));
    if (!P.refresh_measure) return;
    // measurement from the FP64 G just written (this block wrote it; block-wide visibility)
    __threadfence_block();
    __syncthreads();
    const int W = 2 * L + 3;
    uint32_t nmeas = P.nmeas[c];
    const int b = static_cast<int>(nmeas / P.bin_size);
    double* bin = P.bins + (static_cast<size_t>(c) * P.max_bins + b) * W;
    const double* G0 = Gout;
    const double* G1 = Gout + LL;
    for (int m = tid; m < L; m += kT32) {
        double s0 = 0.0, s1 = 0.0;
        for (int q = 0; q < L; ++q) {
            int l = q + m;
            if (l >= L) l -= L;
            int r = l + m;
            const bool wrap = r >= L;
            if (wrap) r -= L;
            const double x0 = G0[r * L + l], x1 = G1[r * L + l];
            s0 = wrap ? s0 - x0 : s0 + x0;
            s1 = wrap ? s1 - x1 : s1 + x1;
        }
        if (b < P.max_bins) {
            bin[m] += s0 / L;
            bin[L + m] += s1 / L;
        }
    }
    double nu = 0.0, nd = 0.0, db = 0.0;
    for (int l = tid; l < L; l += kT32) {
        const double a = 1.0 - G0[l * L + l];
        const double bb = 1.0 - G1[l * L + l];
        nu += a;
        nd += bb;
        db += a * bb;
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
        double a = 0.0, bb = 0.0, cc = 0.0;
        for (int k = 0; k < kT32 / 32; ++k) {
            a += red[k];
            bb += red[8 + k];
            cc += red[16 + k];
        }
        if (b < P.max_bins) {
            bin[2 * L + 0] += a / L;
            bin[2 * L + 1] += bb / L;
            bin[2 * L + 2] += cc / L;
        }
        P.nmeas[c] = nmeas + 1;
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
    refresh_f64_kernel<<<p.nchain, kT32, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace hfk
