// k_lattice_wide.cu -- the lattice step of eq. 2 for bands wider than a shared-memory window
// (the periodic three-dimensional boxes of "Efficient simulations for three dimensions": a
// periodic n^3 box in the folded band order has half-width b = 2 n^2, 392 for 14^3 and 512 for
// 16^3).
//
// Per (w_n, sigma) matrix M = (i w_n + mu) 1 - H0 - diag(Sigma(i w_n)) (complex symmetric, band
// half-width b, no pivoting: the imaginary part of every Schur complement's diagonal stays >= w_n):
//   1. the band of M is written to the matrix's band buffer, column k holding M[k+d][k], d <= b;
//   2. M = L D L^T in place, right-looking and blocked: a panel of kNB columns is staged in shared
//      memory, factored there and written back, and its rank-kNB update of the trailing b x b
//      triangle is applied in the buffer (each entry read and written once per panel);
//   3. G_kk = (M^{-1})_kk = sum_j y_j^2 / D_j with y = L^{-1} e_k (M^{-1} = L^{-T} D^{-1} L^{-1}),
//      by forward substitution from position k, for one listed position per output (orbit, spin
//      slot).  All members of an orbit with the same sublattice relation to its representative
//      have the same G_kk, so the host lists the member with the largest band position: its
//      solve, which runs from k to N - 1, is the shortest.  A solve task takes kR positions at
//      once, each reading of a column of L serving all of them.
// Both run in one persistent kernel (one block per SM) that hands out the factorisations first
// and then the solve tasks, so that the solves fill the SMs the last factorisations leave idle.
// Work per matrix: about N b^2 / 2 complex FMA for the factorisation and (N - k) b per listed
// position, against 1.5 N b^2 for the selected inversion of the window form, which also yields
// every diagonal element.
#include <algorithm>

#include "hf_internal.cuh"

#include "k_lattice.cuh"
#include "k_lattice_dev.cuh"

namespace hfk {
namespace {

constexpr int kNB = 16;          // panel width
constexpr int kT = 512;          // threads of a block (both kinds of task)
constexpr int kR = 16;           // right-hand sides per solve task
constexpr int kWideMaxBand = 840;
constexpr int kSeg = 256;        // rows of a trailing-update unit (8 per lane)

static_assert(kWideMaxBand <= 2 * kT, "two band entries of a column per solve thread at most");

size_t factor_smem(int b) {      // the panel and the pivot row
    return (static_cast<size_t>(kNB) * (kNB + b) + kNB) * sizeof(double2);
}

size_t solve_smem(int b) {       // kR windows of b + 1 entries
    return static_cast<size_t>(kR) * (b + 1) * sizeof(double2);
}

size_t wide_smem(int b) { return std::max(factor_smem(b), solve_smem(b)); }

__device__ __forceinline__ double2 cfma(double2 acc, double2 a, double2 b) {  // acc + a b
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

__device__ __forceinline__ double2 shfl_c(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Matrix qi of the launch: assembly and blocked band L D L^T into its band buffer (column k: D_k
// at d = 0, L_{k+d,k} at d >= 1).  Sets bad on a vanishing or non-finite pivot.
__device__ void factor_matrix(const LatticeArgs& A, int q0, int qi, unsigned char* smem, bool& bad) {
    int sp, n;
    item_of(A, q0 + qi, sp, n);
    const int N = A.N, b = A.b, S = b + 1, RP = kNB + b;
    const int tid = static_cast<int>(threadIdx.x), lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kT / 32;
    const double wn = (2.0 * n + 1.0) * M_PI / A.beta;
    double2* Bq = A.scratch + static_cast<size_t>(qi) * N * S;
    double2* P = reinterpret_cast<double2*>(smem);   // [kNB][RP]: P[j][i] = entry (k0 + i, k0 + j)
    double2* vj = P + static_cast<size_t>(kNB) * RP; // [kNB] pivot row of the current column
    const double2 zero = make_double2(0.0, 0.0);

    // 1. the band of M (entries past the last row zero)
    for (int k = warp; k < N; k += kWarps)
        for (int d = lane; d < S; d += 32) {
            const size_t e = static_cast<size_t>(k) * S + d;
            double2 v = zero;
            if (k + d < N) v = d == 0 ? m_diag(A, k, sp, n, wn) : make_double2(-A.h0band[e], 0.0);
            Bq[e] = v;
        }
    __syncthreads();

    // 2. panels of kNB columns
    for (int k0 = 0; k0 < N; k0 += kNB) {
        const int nb = min(kNB, N - k0);
        const int rmax = min(RP, N - k0);            // rows k0 .. k0 + rmax - 1 exist
        // (a) stage the panel, zero outside each column's band
        for (int j = warp; j < kNB; j += kWarps)
            for (int i = lane; i < RP; i += 32) {
                double2 v = zero;
                if (j < nb && i >= j && i - j <= b && i < rmax)
                    v = Bq[static_cast<size_t>(k0 + j) * S + (i - j)];
                P[j * RP + i] = v;
            }
        __syncthreads();
        // (b) factor it: column j -> L (scaled by 1/D_j); A[i][j'] -= L_ij v_j' (v = D_j L_j'j)
        for (int j = 0; j < nb; ++j) {
            const double2 D = P[j * RP + j];
            if (tid > j && tid < nb) vj[tid] = P[j * RP + tid];
            if (tid == 0 && (!(fabs(D.x) + fabs(D.y) > 0.0) || !isfinite(D.x) || !isfinite(D.y)))
                bad = true;
            __syncthreads();
            const double2 inv = crecip(D);
            for (int i = j + 1 + tid; i < rmax; i += kT) {
                const double2 l = cmul(P[j * RP + i], inv);
                P[j * RP + i] = l;
                const int jm = min(nb - 1, i);
                for (int jp = j + 1; jp <= jm; ++jp) P[jp * RP + i] = cfms(P[jp * RP + i], l, vj[jp]);
            }
            __syncthreads();
        }
        // (c) D and L of the panel back to the buffer
        for (int j = warp; j < nb; j += kWarps) {
            const int ie = min(j + b, rmax - 1);
            for (int i = j + lane; i <= ie; i += 32) Bq[static_cast<size_t>(k0 + j) * S + (i - j)] = P[j * RP + i];
        }
        // (d) trailing triangle, rows and columns nb .. tend (relative to k0):
        //     A[r][c] -= sum_j L_rj w_j with w_j = D_j L_cj; a warp takes a column, 256 rows at a
        //     time (8 a lane); lane j forms w_j once and the warp reads it by shuffle
        const int tend = min(nb - 1 + b, rmax - 1);
        for (int c = nb + warp; c <= tend; c += kWarps) {
            double2* col = Bq + static_cast<size_t>(k0 + c) * S;     // col[r - c]
            const double2 wl = lane < nb ? cmul(P[lane * RP + lane], P[lane * RP + c]) : zero;
            for (int r0 = c; r0 <= tend; r0 += kSeg) {
                const int nqv = min(kSeg / 32, (tend - r0 + 32) >> 5);   // row groups (warp-uniform)
                double2 a[kSeg / 32], acc[kSeg / 32];
#pragma unroll
                for (int q = 0; q < kSeg / 32; ++q) {
                    const int r = r0 + lane + 32 * q;
                    a[q] = (q < nqv && r <= tend) ? col[r - c] : zero;
                    acc[q] = zero;
                }
                for (int j = 0; j < nb; ++j) {
                    const double2 w = shfl_c(wl, j);
                    const double2* pj = P + j * RP;
#pragma unroll
                    for (int q = 0; q < kSeg / 32; ++q)
                        if (q < nqv) acc[q] = cfma(acc[q], pj[min(r0 + lane + 32 * q, tend)], w);
                }
#pragma unroll
                for (int q = 0; q < kSeg / 32; ++q) {
                    const int r = r0 + lane + 32 * q;
                    if (q < nqv && r <= tend) col[r - c] = make_double2(a[q].x - acc[q].x, a[q].y - acc[q].y);
                }
            }
        }
        __syncthreads();
    }
}

// Listed positions ch * kR ... of matrix qi: y = L^{-1} e_p for each position p, in a window of
// b + 1 entries per right-hand side (index j in slot j mod (b + 1)); G_pp = sum_j y_j^2 / D_j.
// The factors were written by another block: they are read through L2 (ld.global.cg).
template <int DPT>   // band entries of a column per thread: b <= DPT * kT
__device__ void solve_chunk(const LatticeArgs& A, int q0, int qi, int ch, unsigned char* smem) {
    int sp, n;
    item_of(A, q0 + qi, sp, n);
    const int N = A.N, b = A.b, S = b + 1;
    const int tid = static_cast<int>(threadIdx.x);
    const double2 zero = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
    const double2* Bq = A.scratch + static_cast<size_t>(qi) * N * S;
    const int* pos = A.wide_pos + static_cast<size_t>(sp) * A.wide_npos + ch * kR;
    const int* out = A.wide_out + static_cast<size_t>(sp) * A.wide_npos + ch * kR;
    const int nr = min(kR, A.wide_npos - ch * kR);
    double2* Y = reinterpret_cast<double2*>(smem);   // [kR][S]
    const int j0 = pos[0];                           // the smallest position of the task
    for (int e = tid; e < kR * S; e += kT) Y[e] = zero;
    __syncthreads();
    int pmine = -1;
    if (tid < nr) {
        pmine = pos[tid];
        if (pmine - j0 < S) Y[tid * S + pmine % S] = one;
    }
    __syncthreads();
    double2 acc = zero;
    int s = j0 % S;
    // column j of L for this thread's entries d = 1 + tid + m kT, loaded a column ahead
    double2 l[DPT];
#pragma unroll
    for (int m = 0; m < DPT; ++m) {
        const int d = 1 + tid + m * kT;
        l[m] = d <= min(b, N - 1 - j0) ? __ldcg(Bq + static_cast<size_t>(j0) * S + d) : zero;
    }
    for (int j = j0; j < N; ++j) {
        const int dmax = min(b, N - 1 - j);
        double2 ln[DPT];
        const int dnext = min(b, N - 2 - j);
#pragma unroll
        for (int m = 0; m < DPT; ++m) {
            const int d = 1 + tid + m * kT;
            ln[m] = d <= dnext ? __ldcg(Bq + static_cast<size_t>(j + 1) * S + d) : zero;
        }
        double2 y[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) y[r] = r < nr ? Y[r * S + s] : zero;
        const double2 ym = tid < nr ? Y[tid * S + s] : zero;
        const double2 Dj = tid < nr ? __ldcg(Bq + static_cast<size_t>(j) * S) : one;
        __syncthreads();                                 // slot s read by every thread
        if (tid < nr) {
            acc = cfma(acc, cmul(ym, ym), crecip(Dj));
            Y[tid * S + s] = (j + S == pmine) ? one : zero;   // the slot now holds index j + S
        }
#pragma unroll
        for (int m = 0; m < DPT; ++m) {
            const int d = 1 + tid + m * kT;
            if (d <= dmax) {
                int sd = s + d;
                if (sd >= S) sd -= S;
#pragma unroll
                for (int r = 0; r < kR; ++r)
                    if (r < nr) Y[r * S + sd] = cfms(Y[r * S + sd], l[m], y[r]);
            }
        }
#pragma unroll
        for (int m = 0; m < DPT; ++m) l[m] = ln[m];
        __syncthreads();
        if (++s == S) s = 0;
    }
    if (tid < nr) {
        A.gloc[static_cast<size_t>(out[tid]) * A.nw + n] = acc;
        if (!isfinite(acc.x) || !isfinite(acc.y)) atomicExch(A.status, static_cast<int>(HF_ENUMERIC));
    }
}

// One persistent block per SM.  The tasks of a launch are the nq factorisations, then the
// nq * nchunk solve tasks (matrix-major); blocks take them in order from work[0].  A block that
// finishes a factorisation raises work[1 + qi]; a solve task waits for its matrix's flag (it was
// handed out earlier, so a running block is factoring it), at most wait_cycles (several times
// what one factorisation takes), after which it reports HF_ETIMEOUT and skips.  So the blocks left over when the factorisations run out take
// the solves of the matrices already factored, instead of idling through a last partial wave.
template <int DPT>
__global__ void __launch_bounds__(kT, 1) lattice_wide_kernel(const LatticeArgs A, int q0, int nq,
                                                             int nchunk, int* work,
                                                             long long wait_cycles) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int task_s, ready_s;
    const int tid = static_cast<int>(threadIdx.x);
    const int ntask = nq * (1 + nchunk);
    bool bad = false;
    for (;;) {
        if (tid == 0) task_s = atomicAdd(work, 1);
        __syncthreads();
        const int t = task_s;
        if (t >= ntask) break;
        if (t < nq) {
            factor_matrix(A, q0, t, smem, bad);
            __syncthreads();                         // every store of the factors issued
            if (tid == 0) {
                __threadfence();
                atomicExch(work + 1 + t, 1);
            }
        } else {
            const int u = t - nq, qi = u / nchunk, ch = u - qi * nchunk;
            if (tid == 0) {
                const long long t0 = clock64();
                int r = load_acquire(work + 1 + qi);
                while (r == 0 && clock64() - t0 < wait_cycles) {
                    __nanosleep(1000);
                    r = load_acquire(work + 1 + qi);
                }
                ready_s = r;
            }
            __syncthreads();
            if (ready_s) solve_chunk<DPT>(A, q0, qi, ch, smem);
            else if (tid == 0) atomicExch(A.status, static_cast<int>(HF_ETIMEOUT));
        }
        __syncthreads();                             // task_s and the shared memory are reused
    }
    if (bad) atomicExch(A.status, static_cast<int>(HF_ENUMERIC));
}

}  // namespace

int lattice_wide_max_band() { return kWideMaxBand; }

int lattice_wide_rhs_per_block() { return kR; }

cudaError_t launch_lattice_wide(const LatticeArgs& a, int q0, int nq, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (a.b < 0 || a.b > kWideMaxBand || a.wide_npos <= 0 || !a.wide_pos || !a.wide_out || !a.work)
        return cudaErrorInvalidValue;
    const bool one = a.b <= kT;
    auto kern = one ? lattice_wide_kernel<1> : lattice_wide_kernel<2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(wide_smem(kWideMaxBand)));
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.work, 0, sizeof(int) * (static_cast<size_t>(nq) + 1), st);
    if (e != cudaSuccess) return e;
    const int nchunk = (a.wide_npos + kR - 1) / kR;
    const int grid = static_cast<int>(std::min<long long>(sms, static_cast<long long>(nq) * (1 + nchunk)));
    // a factorisation takes about N b^2 SM cycles (N b^2 / 2 complex multiply-adds of 4 DFMA at
    // 2 DFMA per cycle); a solve task waits at most 8 times that, and at least 2^31 cycles
    const long long wait = (1ll << 31) + 8ll * a.N * static_cast<long long>(a.b) * a.b;
    kern<<<grid, kT, wide_smem(a.b), st>>>(a, q0, nq, nchunk, a.work, wait);
    return cudaGetLastError();
}

}  // namespace hfk
