// hf_internal.cuh -- shared declarations of the sm_103a Hirsch-Fye QMC / RDMFT library.
//
// Device state of one context lives in a caller-owned workspace; the kernels below are
// launched only by hf_api.cu.  Conventions follow include/hf.h (positive Green functions,
// spin 0 = up).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hf.h"

namespace hfk {

constexpr int kMaxProblems = 16;    // problems fused into one QMC launch
constexpr int kBlock = 128;         // threads per QMC block (4 warps)
constexpr int kMaxL64 = 64;         // largest slice count of the FP64 sweep
constexpr int kMaxL32 = 128;        // largest slice count of the FP32 sweep

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based generator keyed by
// (seed_lo, seed_hi); the counter of proposal (sweep w, slice l) of chain c of site i is
// (w, l, c, i); sweep 0xFFFFFFFF draws the initial fields.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            key.x += 0x9E3779B9u;
            key.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x);
        const uint32_t lo0 = 0xD2511F53u * ctr.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z);
        const uint32_t lo1 = 0xCD9E8D57u * ctr.z;
        ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    }
    return ctr;
}

// 53-bit uniform in [0, 1): ((x << 32 | y) >> 11) * 2^-53.
__device__ __forceinline__ double uniform53(uint4 x) {
    const unsigned long long bits =
        ((static_cast<unsigned long long>(x.x) << 32) | x.y) >> 11;
    return static_cast<double>(bits) * 0x1p-53;
}

// The 53 bits of that uniform as an integer (u = bits * 2^-53).
__device__ __forceinline__ unsigned long long uniform_bits53(uint4 x) {
    return ((static_cast<unsigned long long>(x.x) << 32) | x.y) >> 11;
}

// 24-bit uniform in [0, 1) for the single-precision sweep: (x >> 8) * 2^-24.
__device__ __forceinline__ float uniform24(uint4 x) {
    return static_cast<float>(x.x >> 8) * 0x1p-24f;
}

// ---------------------------------------------------------------------------------------
// One QMC problem (one context) as seen by the fused sweep kernel.
// ---------------------------------------------------------------------------------------
struct QmcProblem {
    int L;                // time slices
    int cps;              // chains per inequivalent site
    int nchain;           // chains of this problem
    int block0;           // first block of this problem in the launch
    uint32_t seed_lo, seed_hi;
    double a_p, a_m;      // e^{-2 lambda} - 1 (sigma s_l = +1), e^{+2 lambda} - 1 (= -1)
    double ev_p, ev_m;    // e^{+lambda} - 1, e^{-lambda} - 1 (Dyson factors, sigma s = +-1)
    float af_p, af_m;     // single-precision copies of a_p, a_m (rounded to nearest)
    float afl_p, afl_m;   // remainders: a_p ~ af_p + afl_p as a double-float
    int n_warmup, n_measure, refresh_every, bin_size, max_bins, refresh_first;
    // single-precision path only: sweeps of this launch and the measured local range
    int nsweeps, meas_from, meas_to;
    int refresh_measure;  // refresh kernel: add a measurement after the refresh
    int team_warps;       // FP64 / FP32-pair sweeps: warps per chain (1, 2, 4; >= 2 for L > 32)
    int site0;            // Philox site word = site0 + local site (served requests: the key's site)
    int delay_k;          // FP32-pair sweeps: delayed-update depth (<= 1: rank-1 updates)
    int refresh_stagger;  // 1: chain (site, c) refreshes when nsw + site + c = 0 mod refresh_every
    int slot_mult;        // FP64 / FP32-pair sweeps: block slot s runs chain (s slot_mult) mod
                          // nchain (gcd(slot_mult, nchain) = 1), so that a block's chains come
                          // from sites across the trap and blocks carry similar work; 1: slot s
                          // runs chain s
    const double* gtau;   // [nsite][2][L]  bath g~0(tau_m)
    double* g0inv;        // [nsite][2][L*L] inverse bath matrices (rebuilt with the bath)
    double* G;            // [nchain][2][L*L] (FP64 state, or FP64 scratch of the FP32 path)
    float* Gf;            // [nchain][2][L*L] FP32 state (precision 1) or nullptr
    int8_t* s;            // [nchain][L]
    uint32_t* nsw;        // [nchain] sweeps done
    uint32_t* nmeas;      // [nchain] measurements since the last clear
    unsigned long long* acc;  // [nchain] accepted flips
    double* bins;         // [nchain][max_bins][2L+3]
    int* status;          // [0]: error code (HF_ENUMERIC...), [1]: non-positive ratios seen
    unsigned int* drift;  // nullptr, or [0] largest |G_SM - G_Dyson| met at an in-launch refresh
                          // (float bits) and [1] refreshes checked
};

struct QmcBatch {
    int nprob;
    int nblocks;
    QmcProblem p[kMaxProblems];
};

// Drift monitor: folds the largest |G_SM - G_Dyson| v >= 0 a warp has seen into the context's
// words -- [0] the maximum as float bits (non-negative floats order like their bit patterns, so an
// integer maximum keeps the float maximum), [1] one count per chain refresh (count = true on one
// thread of the team).  Every lane of the warp takes part.
__device__ __forceinline__ void drift_fold(unsigned int* drift, float v, bool count) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(drift, __float_as_uint(v));
    if (count) atomicAdd(drift + 1, 1u);
}

// FP64 and FP32-pair sweeps: blocks of kBlock threads hold 4 / team_warps chains.
size_t qmc_f64_smem_bytes(int L, int team_warps);
bool qmc_f64_supported(int L);
cudaError_t launch_qmc_f64(const QmcBatch& b, size_t smem, cudaStream_t st);
int qmc_f64_chains_per_block(int L, int team_warps);
int qmc_default_team_warps(int L);

// FP32-pair ("double-float") sweeps with FP64 refresh: same layout and L set as the FP64 kernel.
cudaError_t launch_qmc_df64(const QmcBatch& b, size_t smem, cudaStream_t st);
size_t qmc_df64_smem_bytes(int L, int team_warps, int delay_k);

size_t qmc_f32_smem_bytes(int L);
bool qmc_f32_supported(int L);
cudaError_t launch_qmc_f32(const QmcBatch& b, size_t smem, cudaStream_t st);
int qmc_f32_chains_per_block(int L);
// FP64 Dyson refresh of every chain of one problem (L <= 128): writes G (FP64) and, when
// p.Gf is set, its FP32 copy; measures afterwards when p.refresh_measure is set.
size_t refresh_f64_smem_bytes(int L);
cudaError_t launch_refresh_f64(const QmcProblem& p, cudaStream_t st);
// g0^{-1} of every (site, spin) of every problem of b, from p.gtau into p.g0inv (nchain / cps
// sites each); the refreshes of all three sweep forms read it, so it is rebuilt whenever a bath
// changes.
cudaError_t launch_g0_inverse(const QmcBatch& b, cudaStream_t st);

cudaError_t launch_init_fields(int8_t* s, int nchain, int cps, int L, uint32_t seed_lo,
                               uint32_t seed_hi, cudaStream_t st, int site0 = 0);

// Reduction of bins over chains: out_mean/out_err [nsite][2L+4].
cudaError_t launch_reduce(const double* bins, int nsite, int cps, int L, int max_bins,
                          int nbins_done, int bin_size, double* out_mean, double* out_err,
                          cudaStream_t st);

}  // namespace hfk
