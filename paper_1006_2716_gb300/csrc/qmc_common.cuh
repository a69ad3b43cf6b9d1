// qmc_common.cuh -- device helpers shared by the FP64 and FP32-pair Hirsch-Fye sweep kernels:
// team synchronisation, the per-chain shared-memory layout, integer-pipe FP32/FP64 views, the
// Newton reciprocal and the FP64 Dyson refresh (G = M^{-1}, M = g0^{-1} e^V - (e^V - 1), by
// in-place Gauss-Jordan elimination with partial pivoting in shared memory).
#pragma once

#include "hf_internal.cuh"

namespace hfk {
namespace qmc {

// A team of TW warps owns one chain; a 128-thread block holds 4 / TW teams.  One-warp teams
// synchronise with __syncwarp, the whole-block team with __syncthreads, two-warp teams with the
// named barrier 1 + team index over their 64 threads.  Every call site is reached by all threads
// of the team in the same order (the control flow around it depends only on shared data that
// all of them read before any thread of the team writes it); the explicit __syncwarp
// reconverges the warp, since the compiler does not treat inline assembly as a barrier, so the
// aligned form of the named barrier applies.
template <int TW>
__device__ __forceinline__ void team_sync() {
    if constexpr (TW == 1) {
        __syncwarp();
    } else if constexpr (TW * 32 == kBlock) {
        __syncthreads();
    } else {
        __syncwarp();
        asm volatile("bar.sync %0, %1;" ::"r"(1 + static_cast<int>(threadIdx.x) / (32 * TW)),
                     "r"(32 * TW)
                     : "memory");
    }
}

// Shared-memory footprint of one team (bytes), rounded up to 16 bytes so that every team of a
// block starts 16-byte aligned.
__host__ __device__ constexpr size_t team_bytes(int L) {
    return (static_cast<size_t>(2 * L * L + 7 * L + 11) * 8 + 16 + ((L + 15) / 16) * 16 + 15) /
           16 * 16;
}

template <int L>
struct TeamSmem {
    double* G0;    // [L*L]
    double* G1;    // [L*L]
    double* cr;    // [4L]: scaled column up/down, row up/down; refresh: multipliers, 1/pivot
    unsigned long long* ub;  // [L] 53-bit uniforms as integers
    double* bacc;  // [2L+3] current bin
    double* red;   // [8]
    int* piv;      // [4]
    int8_t* s;     // [L]
    __device__ explicit TeamSmem(unsigned char* base) {
        double* d = reinterpret_cast<double*>(base);
        G0 = d;
        G1 = G0 + L * L;
        cr = G1 + L * L;
        ub = reinterpret_cast<unsigned long long*>(cr + 4 * L);
        bacc = reinterpret_cast<double*>(ub + L);
        red = bacc + 2 * L + 3;
        piv = reinterpret_cast<int*>(red + 8);
        s = reinterpret_cast<int8_t*>(piv + 4);
    }
};

// |x| ordering through the bit pattern (integer pipe): larger magnitude -> larger key.
__device__ __forceinline__ unsigned long long mag_key(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
}

// Single-precision view of a double built on the integer pipe from its bit pattern (mantissa
// truncated to 23 bits, |relative error| < 2^-23; magnitudes outside the float range flush
// to 0 or saturate to FLT_MAX, which only widens the decision guard below).
__device__ __forceinline__ float f32_of(double x) {
    const int hi = __double2hiint(x);
    const unsigned lo = static_cast<unsigned>(__double2loint(x));
    const int e = ((hi >> 20) & 0x7FF) - 1023 + 127;
    const unsigned sign = static_cast<unsigned>(hi) & 0x80000000u;
    const unsigned mant = ((static_cast<unsigned>(hi) & 0xFFFFFu) << 3) | (lo >> 29);
    if (e <= 0) return __int_as_float(static_cast<int>(sign));
    if (e >= 255) return __int_as_float(static_cast<int>(sign | 0x7F7FFFFFu));
    return __int_as_float(static_cast<int>(sign | (static_cast<unsigned>(e) << 23) | mant));
}

// Double from a (normal, nonzero) float's bit pattern, integer pipe only.
__device__ __forceinline__ double f64_of(float f) {
    const unsigned b = static_cast<unsigned>(__float_as_int(f));
    const unsigned sign = b & 0x80000000u;
    const unsigned e = ((b >> 23) & 0xFFu) + (1023u - 127u);
    const unsigned mant = b & 0x7FFFFFu;
    return __hiloint2double(static_cast<int>(sign | (e << 20) | (mant >> 3)),
                            static_cast<int>(mant << 29));
}

// 1/R to ~1 ulp: FP32 reciprocal seed (22 bits) and two Newton steps in FP64 (4 DFMA)
// instead of a full IEEE division.  R is a flip ratio: finite, normal, |R| well inside the float
// range.
__device__ __forceinline__ double recip64(double R, float Rf) {
    double r = f64_of(__frcp_rn(Rf));
    double e = fma(-R, r, 1.0);
    r = fma(r, e, r);
    e = fma(-R, r, 1.0);
    return fma(r, e, r);
}

// Dyson refresh by way of the inverse Green function.  A G = g0 with A = 1 + (1 - g0) D,
// D = diag(e^{V_j} - 1), gives G^{-1} = g0^{-1} A = g0^{-1} e^V - D, so with g0^{-1} computed
// once per bath a refresh is one inversion of M = g0^{-1} e^V - D: L^3 FP64 multiply-adds per
// spin against the (4/3) L^3 of factoring A and solving for the L columns of g0.

// The bath matrix itself, g0[l][l'] = g~0(tau_l - tau_l') (negated for l < l'): at U = 0 every
// e^{V_j} is 1, A = 1 and the Dyson relation gives G = g0 exactly, with no inversion.
template <int L, int TW>
__device__ void build_bath_matrix(const double* gt, double* G, int tid) {
    constexpr int T = 32 * TW;
    for (int e = tid; e < L * L; e += T) {
        const int i = e / L, j = e - (e / L) * L;
        const int d = i - j;
        G[e] = (d >= 0) ? gt[d] : -gt[d + L];
    }
}

// M[i][j] = g0inv[i][j] e^{V_j} - delta_ij (e^{V_j} - 1), V_j = lambda sigma s_j (dense, row-major)
template <int L, int TW>
__device__ void build_inverse_dyson(const QmcProblem& P, const double* g0inv, const int8_t* s,
                                    int sigma, double* M, int tid) {
    constexpr int T = 32 * TW;
    for (int e = tid; e < L * L; e += T) {
        const int i = e / L, j = e - (e / L) * L;
        const bool up = sigma * s[j] > 0;
        const double ev = up ? P.ev_p : P.ev_m;
        const double m = g0inv[e] * (1.0 + ev);
        M[e] = (i == j) ? m - ev : m;
    }
}

// In-place inverse of the dense row-major L x L matrix M by Gauss-Jordan elimination with partial
// pivoting by rows, by a team of 32 TW threads: step k takes the largest |M[i][k]|, i >= k, as
// pivot (the smallest i among equal magnitudes), swaps it into row k, scales row k by its
// reciprocal, moves column k out and subtracts its multiples of row k from every other row; the
// column order is restored at the end.  Scratch: fcol[L] doubles, pivrow[L] ints, flag[2] ints,
// *pinv.  Returns false if a pivot column was exactly zero.
template <int L, int TW>
__device__ bool gj_team(double* M, double* fcol, int* pivrow, int* flag, double* pinv, int tid) {
    constexpr int T = 32 * TW;
    bool ok = true;
    for (int k = 0; k < L; ++k) {
        if (tid < 32) {
            unsigned long long best = 0ull;
            int bi = L;
            for (int i = k + tid; i < L; i += 32) {
                const unsigned long long key = mag_key(M[i * L + k]);
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
                pivrow[k] = bi;
                flag[0] = bi;
                flag[1] = (best == 0ull) ? 1 : 0;
                *pinv = 1.0 / M[bi * L + k];
            }
        }
        team_sync<TW>();
        const int p = flag[0];
        if (flag[1]) ok = false;
        if (p != k) {
            for (int j = tid; j < L; j += T) {
                const double t = M[k * L + j];
                M[k * L + j] = M[p * L + j];
                M[p * L + j] = t;
            }
            team_sync<TW>();
        }
        const double pv = *pinv;
        // disjoint elements: row k (scaled; its diagonal becomes the reciprocal) and the rest of
        // column k (copied out and zeroed)
        for (int j = tid; j < L; j += T) {
            const double x = M[k * L + j];
            M[k * L + j] = (j == k) ? pv : x * pv;
        }
        for (int i = tid; i < L; i += T) {
            if (i != k) {
                fcol[i] = M[i * L + k];
                M[i * L + k] = 0.0;
            } else {
                fcol[i] = 0.0;
            }
        }
        team_sync<TW>();
        for (int e = tid; e < L * L; e += T) {
            const int i = e / L, j = e - (e / L) * L;
            if (i != k) M[e] = fma(-fcol[i], M[k * L + j], M[e]);
        }
        team_sync<TW>();
    }
    for (int k = L - 1; k >= 0; --k) {   // undo the row swaps as column swaps, last first
        const int p = pivrow[k];
        if (p != k) {
            for (int i = tid; i < L; i += T) {
                const double t = M[i * L + k];
                M[i * L + k] = M[i * L + p];
                M[i * L + p] = t;
            }
            team_sync<TW>();
        }
    }
    team_sync<TW>();   // every thread has read pivrow before the scratch is reused
    return ok;
}

// Scratch of gj_team inside a team's shared memory: fcol = cr[0..L), *pinv = cr[L], pivrow in
// the ints from cr + L + 1 on (L ints fit in the remaining 3L - 1 doubles), flag = piv[0..1].
template <int L>
struct GjTeamScratch {
    double* fcol;
    double* pinv;
    int* pivrow;
    int* flag;
    __device__ explicit GjTeamScratch(const TeamSmem<L>& S)
        : fcol(S.cr), pinv(S.cr + L), pivrow(reinterpret_cast<int*>(S.cr + L + 1)), flag(S.piv) {}
};

}  // namespace qmc
}  // namespace hfk
