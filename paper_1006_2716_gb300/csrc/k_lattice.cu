// k_lattice.cu -- RDMFT lattice step on sm_103a (eq. 2 of the paper).
//
//   G(i w_n) = [(i w_n + mu) 1 - H0 - diag(Sigma_sigma(i w_n))]^{-1},  keep G_ii of the
//   inequivalent sites.  Frequencies are independent ("Model and Methods": the inversions for
//   the 500 Matsubara frequencies run in parallel), so one warp owns one (w_n, sigma) matrix.
//
// The paper inverts dense matrices, which it names as the cost that dominates beyond ~1000
// sites.  On a lattice numbered row by row, H0 (nearest-neighbour hopping plus the trap) is a
// band matrix of half-width b (b = Lx for a square; the longest row for the disc), and only the
// diagonal of the inverse is needed.  So each warp
//   1. factors the complex-symmetric band matrix M = L D L^T without pivoting (M has a positive
//      definite imaginary part w_n - Im Sigma >= w_n > 0 on the diagonal, which every Schur
//      complement inherits, so no pivot vanishes), storing L and D in a global band buffer,
//   2. runs the selected-inversion recurrence backwards,
//        Z_ik = -sum_{j in (k, k+b]} Z_ij L_jk   (i in (k, k+b]),
//        Z_kk = 1/D_k - sum_{i in (k, k+b]} L_ik Z_ik,
//      which only touches entries of Z = M^{-1} inside the band, kept as a b x b window in
//      shared memory.
// Work per matrix ~1.5 N b^2 complex FMA instead of the dense (4/3) N^3.
#include <algorithm>

#include "hf_internal.cuh"
#include "k_lattice.cuh"

namespace hfk {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfms(double2 acc, double2 a, double2 b) {  // acc - a b
    return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)),
                        fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 crecip(double2 a) {
    const double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}

__global__ void lattice_kernel(const LatticeArgs A, int q0, int nq) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int qi = blockIdx.x * wpb + warp;    // matrix within this chunk
    if (qi >= nq) return;
    const int q = q0 + qi;                     // q = sigma * nw + n
    const int sp = q / A.nw;
    const int n = q - sp * A.nw;
    const int N = A.N, b = A.b, bw = A.b + 1;
    const double wn = (2.0 * n + 1.0) * M_PI / A.beta;
    double2* F = A.scratch + static_cast<size_t>(qi) * N * bw;   // F[k*bw + d] = M[k+d][k]
    double2* Zw = reinterpret_cast<double2*>(smem) + static_cast<size_t>(warp) * (b * b + 2 * bw);
    double2* lcol = Zw + b * b;        // [bw] L_{k+d,k}
    double2* zcol = lcol + bw;         // [bw] new Z_{k+d,k}

    // 1. assemble the lower band of M
    for (int k = 0; k < N; ++k) {
        for (int d = lane; d < bw; d += 32) {
            double2 v;
            if (d == 0) {
                const int r = A.rep_of[k];
                const int s2 = sp ^ A.flip[k];
                const double2 sg = A.sigma[(static_cast<size_t>(r) * 2 + s2) * A.nw + n];
                v = make_double2(A.mu - A.h0band[static_cast<size_t>(k) * bw] - sg.x, wn - sg.y);
            } else {
                v = make_double2((k + d < N) ? -A.h0band[static_cast<size_t>(k) * bw + d] : 0.0,
                                 0.0);
            }
            F[static_cast<size_t>(k) * bw + d] = v;
        }
    }
    __syncwarp();

    // 2. right-looking band LDL^T
    bool bad = false;
    for (int k = 0; k < N; ++k) {
        const int dmax = min(b, N - 1 - k);
        for (int d = lane; d <= dmax; d += 32) lcol[d] = F[static_cast<size_t>(k) * bw + d];
        __syncwarp();
        const double2 Dk = lcol[0];
        const double2 inv = crecip(Dk);
        if (!(fabs(Dk.x) + fabs(Dk.y) > 0.0) || !isfinite(Dk.x) || !isfinite(Dk.y)) bad = true;
        // L column, stored in place of M's column (D_k stays on the diagonal slot)
        for (int d = 1 + lane; d <= dmax; d += 32) {
            const double2 l = cmul(lcol[d], inv);
            zcol[d] = l;
            F[static_cast<size_t>(k) * bw + d] = l;
        }
        __syncwarp();
        // trailing update: M[k+d1][k+d2] -= L_{k+d1,k} D_k L_{k+d2,k} = L_{k+d1,k} v_d2
        for (int d2 = 1; d2 <= dmax; ++d2) {
            const double2 v2 = lcol[d2];
            for (int d1 = d2 + lane; d1 <= dmax; d1 += 32) {
                double2* t = F + static_cast<size_t>(k + d2) * bw + (d1 - d2);
                *t = cfms(*t, zcol[d1], v2);
            }
        }
        __syncwarp();
    }

    // 3. selected inversion, k = N-1 .. 0; window slot of index i is i mod b
    for (int k = N - 1; k >= 0; --k) {
        const int dmax = min(b, N - 1 - k);
        for (int d = lane; d <= dmax; d += 32) lcol[d] = F[static_cast<size_t>(k) * bw + d];
        __syncwarp();
        // Z_{k+d,k} = -sum_{e=1..dmax} Z_{k+d,k+e} L_{k+e,k}
        for (int d = 1 + lane; d <= dmax; d += 32) {
            const int si = (k + d) % b;
            double2 acc = make_double2(0.0, 0.0);
            for (int e = 1; e <= dmax; ++e) {
                const int sj = (k + e) % b;
                acc = cfms(acc, Zw[si * b + sj], lcol[e]);
            }
            zcol[d] = acc;
        }
        __syncwarp();
        // Z_kk = 1/D_k - sum_d L_{k+d,k} Z_{k+d,k}
        double2 part = make_double2(0.0, 0.0);
        for (int d = 1 + lane; d <= dmax; d += 32) part = cfms(part, lcol[d], zcol[d]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
            part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
        }
        const double2 zkk = make_double2(crecip(lcol[0]).x + part.x, crecip(lcol[0]).y + part.y);
        // insert row/column k into the window (slot of k = slot of the evicted k + b)
        if (b > 0) {
            const int sk = k % b;
            for (int d = 1 + lane; d <= dmax; d += 32) {
                const int si = (k + d) % b;
                Zw[sk * b + si] = zcol[d];
                Zw[si * b + sk] = zcol[d];
            }
            if (lane == 0) Zw[sk * b + sk] = zkk;
        }
        __syncwarp();
        const int r = A.site_rep[k];
        if (r >= 0 && lane == 0)
            A.gloc[(static_cast<size_t>(r) * 2 + sp) * A.nw + n] = zkk;
        if (!isfinite(zkk.x) || !isfinite(zkk.y)) bad = true;
    }
    if (bad && lane == 0) atomicExch(A.status, static_cast<int>(HF_ENUMERIC));
}

}  // namespace

size_t lattice_smem_per_warp(int b) {
    return static_cast<size_t>(b * b + 2 * (b + 1)) * sizeof(double2);
}

bool lattice_band_supported(int b) {
    return b >= 0 && lattice_smem_per_warp(b) <= static_cast<size_t>(227) * 1024;
}

int lattice_max_band() {
    int b = 0;
    while (lattice_band_supported(b + 1)) ++b;
    return b;
}

int lattice_warps_per_block(int b) {
    const size_t per = lattice_smem_per_warp(b);
    int w = 4;
    while (w > 1 && per * w > 200 * 1024) --w;
    return w;
}

size_t lattice_scratch_per_matrix(int N, int b) {
    return static_cast<size_t>(N) * (b + 1) * sizeof(double2);
}

cudaError_t launch_lattice(const LatticeArgs& a, int q0, int nq, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    const int wpb = lattice_warps_per_block(a.b);
    const size_t smem = lattice_smem_per_warp(a.b) * wpb;
    cudaError_t e = cudaFuncSetAttribute(lattice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int blocks = (nq + wpb - 1) / wpb;
    lattice_kernel<<<blocks, 32 * wpb, smem, st>>>(a, q0, nq);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Allocation-free variant: the band buffers live in a fixed device array of this file instead
// of the caller's workspace.  Every GPU that loads the library holds the array until exit.
// Each launch of the kernel overwrites every band element it later reads (step 1 assembles the
// whole band), so nothing left over from an earlier call needs clearing; two calls that overlap
// on the GPU would share the array and race.
// ---------------------------------------------------------------------------------------
constexpr size_t kStaticLatticeScratchBytes = static_cast<size_t>(16) << 20;   // 16 MiB
static __device__ __align__(256) double2
    g_lattice_scratch[kStaticLatticeScratchBytes / sizeof(double2)];

size_t lattice_static_scratch_bytes() { return kStaticLatticeScratchBytes; }

// Device address of g_lattice_scratch on the current device, looked up once per device (the
// host-side symbol is only a stand-in and must never reach a kernel).
static cudaError_t static_scratch_address(double2** out) {
    constexpr int kMaxDevices = 64;
    static double2* addr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_lattice_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = static_cast<double2*>(p);
    }
    *out = addr[dev];
    return cudaSuccess;
}

cudaError_t launch_lattice_static(const LatticeArgs& a_in, cudaStream_t st) {
    const size_t per = lattice_scratch_per_matrix(a_in.N, a_in.b);
    if (per == 0 || per > kStaticLatticeScratchBytes) return cudaErrorInvalidValue;
    double2* base = nullptr;
    cudaError_t e = static_scratch_address(&base);
    if (e != cudaSuccess) return e;
    LatticeArgs a = a_in;
    a.scratch = base;
    const int chunk = static_cast<int>(kStaticLatticeScratchBytes / per);
    const int nq = 2 * a.nw;
    for (int q0 = 0; q0 < nq; q0 += chunk) {
        e = launch_lattice(a, q0, std::min(chunk, nq - q0), st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hfk
