// k_lattice.cu -- RDMFT lattice step on sm_103a (eq. 2 of the paper).
//
//   G(i w_n) = [(i w_n + mu) 1 - H0 - diag(Sigma_sigma(i w_n))]^{-1},  keep G_ii of the
//   inequivalent sites.  Frequencies are independent ("Model and Methods": the inversions for
//   the 500 Matsubara frequencies run in parallel), so each (w_n, sigma) matrix is one work item.
//
// The paper inverts dense matrices, which it names as the cost that dominates beyond ~1000
// sites.  In the band order of the host (rows of the square or disc; folded periodic axes; the
// slab's layers innermost) H0 -- nearest-neighbour hopping plus the trap -- is a band matrix of
// half-width b, and only the diagonal of the inverse is needed.  So each work item
//   1. factors the complex-symmetric band matrix M = L D L^T without pivoting (M has a positive
//      definite imaginary part w_n - Im Sigma >= w_n > 0 on the diagonal, which every Schur
//      complement inherits, so no pivot vanishes),
//   2. runs the selected-inversion recurrence backwards,
//        Z_ik = -sum_{j in (k, k+b]} Z_ij L_jk   (i in (k, k+b]),
//        Z_kk = 1/D_k - sum_{i in (k, k+b]} L_ik Z_ik,
//      which only touches entries of Z = M^{-1} inside the band.
// Work per matrix ~1.5 N b^2 complex FMA instead of the dense (4/3) N^3.
//
// Spin halving: when a symmetry of the lattice exchanges the two sublattices, the self-energy
// built from the orbits satisfies Sigma_{i,dn} = Sigma_{g(i),up}, so M_dn is M_up with its sites
// permuted by g and G_{r,dn} = G_{g(r),up}.  The host then asks for the spin-up matrices only
// (nspin = 1) and names, per band position, the representative whose spin-down value sits there
// (site_dn).
//
// A single packed symmetric window of b + 1 slots in shared memory (index i in slot i mod (b+1))
// holds the active trailing block of the factorisation and then the window of Z; L and D go to
// global memory once and are read back once.  A narrow band (b <= kNarrowBand) takes one warp per
// matrix; a wide one a block of kWideThreads, so that the four schedulers of an SM all issue FP64
// work (this GPU executes 2 FP64 FMA lanes per clock per SM).
#include <algorithm>

#include "hf_internal.cuh"
#include "k_lattice.cuh"

namespace hfk {
namespace {

constexpr int kNarrowBand = 32;
constexpr int kWideThreads = 128;
constexpr int kWideWarps = kWideThreads / 32;

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
__device__ __forceinline__ double2 shfl_xor_c(double2 v, int o) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Matrix q of the launch: spin and Matsubara index.
__device__ __forceinline__ void item_of(const LatticeArgs& A, int q, int& sp, int& n) {
    sp = q / A.nw;
    n = q - sp * A.nw;
}

// Diagonal element of M at band position k.
__device__ __forceinline__ double2 m_diag(const LatticeArgs& A, int k, int sp, int n, double wn) {
    const int bw = A.b + 1;
    const int r = A.rep_of[k];
    const int s2 = sp ^ A.flip[k];
    const double2 sg = A.sigma[(static_cast<size_t>(r) * 2 + s2) * A.nw + n];
    return make_double2(A.mu - A.h0band[static_cast<size_t>(k) * bw] - sg.x, wn - sg.y);
}

// Writes the diagonal G_kk of the matrix to the outputs that take it.
__device__ __forceinline__ void store_diag(const LatticeArgs& A, int k, int sp, int n, double2 z) {
    const int r = A.site_rep[k];
    if (r >= 0) A.gloc[(static_cast<size_t>(r) * 2 + sp) * A.nw + n] = z;
    if (A.site_dn) {
        const int r2 = A.site_dn[k];
        if (r2 >= 0) A.gloc[(static_cast<size_t>(r2) * 2 + 1) * A.nw + n] = z;
    }
}

// Packed symmetric window: the entry of slots (a, c) lives at tri(max, min).
__device__ __forceinline__ int wtri(int a, int c) {
    const int hi = max(a, c), lo = min(a, c);
    return hi * (hi + 1) / 2 + lo;
}

// Element M[i][j] (i >= j, i - j <= b) of the unfactored matrix.
__device__ __forceinline__ double2 m_entry(const LatticeArgs& A, int i, int j, int sp, int n,
                                           double wn) {
    if (i == j) return m_diag(A, i, sp, n, wn);
    return make_double2(-A.h0band[static_cast<size_t>(j) * (A.b + 1) + (i - j)], 0.0);
}

template <int WPM>
__device__ __forceinline__ void mat_sync() {
    if constexpr (WPM == 1) __syncwarp(); else __syncthreads();
}

// One matrix per WPM warps (WPM = 1: several matrices per block, one per warp; WPM = 4: one per
// block).  WPM = 4 spreads rows over the warps and columns over the lanes; WPM = 1 gives each
// lane whole rows, so that no reductions are needed on the short rows of a narrow band.
template <int WPM>
__global__ void __launch_bounds__(128) lattice_kernel(const LatticeArgs A, int q0, int nq) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int T = 32 * WPM;
    const int tid = threadIdx.x % T;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int mi = threadIdx.x / T;
    const int qi = blockIdx.x * (blockDim.x / T) + mi;
    if (qi >= nq) return;      // WPM = 1 only (one matrix per block otherwise)
    int sp, n;
    item_of(A, q0 + qi, sp, n);
    const int N = A.N, b = A.b, S = A.b + 1;
    const double wn = (2.0 * n + 1.0) * M_PI / A.beta;
    double2* Lg = A.scratch + static_cast<size_t>(qi) * N * S;    // Lg[k*S] = D_k, [k*S+d] = L_{k+d,k}
    double2* W = reinterpret_cast<double2*>(smem) + static_cast<size_t>(mi) * (S * (S + 1) / 2 + 2 * S);
    double2* lv = W + S * (S + 1) / 2;                              // [S]
    double2* vv = lv + S;                                           // [S]
    bool bad = false;

    // 1. the window starts as the leading (b+1) x (b+1) block of M (slot = index)
    const int n0 = min(S, N);
    for (int t = tid; t < n0 * (n0 + 1) / 2; t += T) {
        int i = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while (i * (i + 1) / 2 > t) --i;
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        W[t] = m_entry(A, i, t - i * (i + 1) / 2, sp, n, wn);
    }
    mat_sync<WPM>();

    // 2. band LDL^T, right-looking, on the window
    for (int k = 0; k < N; ++k) {
        const int dmax = min(b, N - 1 - k);
        const int sk = k % S;
        const double2 Dk = W[wtri(sk, sk)];
        const double2 inv = crecip(Dk);
        for (int d = 1 + tid; d <= dmax; d += T) {
            const double2 v = W[wtri((k + d) % S, sk)];
            const double2 l = cmul(v, inv);
            vv[d] = v;
            lv[d] = l;
            Lg[static_cast<size_t>(k) * S + d] = l;
        }
        if (tid == 0) {
            Lg[static_cast<size_t>(k) * S] = Dk;
            if (!(fabs(Dk.x) + fabs(Dk.y) > 0.0) || !isfinite(Dk.x) || !isfinite(Dk.y)) bad = true;
        }
        mat_sync<WPM>();
        // trailing update M[k+d1][k+d2] -= L_{k+d1,k} v_d2 (1 <= d2 <= d1 <= dmax)
        if constexpr (WPM == 1) {
            for (int d1 = 1 + lane; d1 <= dmax; d1 += 32) {
                const int s1 = (k + d1) % S;
                const double2 l1 = lv[d1];
                for (int d2 = 1; d2 <= d1; ++d2) {
                    double2* t = W + wtri(s1, (k + d2) % S);
                    *t = cfms(*t, l1, vv[d2]);
                }
            }
        } else {
            for (int d1 = 1 + warp; d1 <= dmax; d1 += WPM) {
                const int s1 = (k + d1) % S;
                const double2 l1 = lv[d1];
                for (int d2 = 1 + lane; d2 <= d1; d2 += 32) {
                    double2* t = W + wtri(s1, (k + d2) % S);
                    *t = cfms(*t, l1, vv[d2]);
                }
            }
        }
        // index k + b + 1 enters the slot of k: its row of the unfactored matrix
        const int inew = k + S;
        if (inew < N)
            for (int j = k + 1 + tid; j <= inew; j += T) W[wtri(sk, j % S)] = m_entry(A, inew, j, sp, n, wn);
        mat_sync<WPM>();
    }

    // 3. selected inversion, k = N-1 .. 0; the window now holds Z for the indices in (k, k+b]
    for (int k = N - 1; k >= 0; --k) {
        const int dmax = min(b, N - 1 - k);
        const int sk = k % S;
        for (int e = 1 + tid; e <= dmax; e += T) lv[e] = Lg[static_cast<size_t>(k) * S + e];
        mat_sync<WPM>();
        // Z_{k+d,k} = -sum_e Z_{k+d,k+e} L_{k+e,k}
        if constexpr (WPM == 1) {
            for (int d = 1 + lane; d <= dmax; d += 32) {
                const int s1 = (k + d) % S;
                double2 acc = make_double2(0.0, 0.0);
                for (int e = 1; e <= dmax; ++e) acc = cfms(acc, W[wtri(s1, (k + e) % S)], lv[e]);
                vv[d] = acc;
            }
        } else {
            for (int d = 1 + warp; d <= dmax; d += WPM) {
                const int s1 = (k + d) % S;
                double2 acc = make_double2(0.0, 0.0);
                for (int e = 1 + lane; e <= dmax; e += 32) acc = cfms(acc, W[wtri(s1, (k + e) % S)], lv[e]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double2 t = shfl_xor_c(acc, o);
                    acc.x += t.x;
                    acc.y += t.y;
                }
                if (lane == 0) vv[d] = acc;
            }
        }
        mat_sync<WPM>();
        // row/column k into the slot of k (which held k + b + 1, outside every later window)
        for (int d = 1 + tid; d <= dmax; d += T) W[wtri(sk, (k + d) % S)] = vv[d];
        if (warp == 0) {
            double2 part = make_double2(0.0, 0.0);
            for (int d = 1 + lane; d <= dmax; d += 32) part = cfms(part, lv[d], vv[d]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double2 t = shfl_xor_c(part, o);
                part.x += t.x;
                part.y += t.y;
            }
            if (lane == 0) {
                const double2 ri = crecip(Lg[static_cast<size_t>(k) * S]);
                const double2 zkk = make_double2(ri.x + part.x, ri.y + part.y);
                W[wtri(sk, sk)] = zkk;
                store_diag(A, k, sp, n, zkk);
                if (!isfinite(zkk.x) || !isfinite(zkk.y)) bad = true;
            }
        }
        mat_sync<WPM>();
    }
    if (bad) atomicExch(A.status, static_cast<int>(HF_ENUMERIC));
}

size_t window_bytes(int b) {     // one matrix: packed window and two vectors
    const size_t S = static_cast<size_t>(b) + 1;
    return (S * (S + 1) / 2 + 2 * S) * sizeof(double2);
}

}  // namespace

bool lattice_band_supported(int b) {
    return b >= 0 && window_bytes(b) <= static_cast<size_t>(227) * 1024;
}

int lattice_max_band() {
    int b = 0;
    while (lattice_band_supported(b + 1)) ++b;
    return b;
}

size_t lattice_scratch_per_matrix(int N, int b) {
    return static_cast<size_t>(N) * (b + 1) * sizeof(double2);
}

cudaError_t launch_lattice(const LatticeArgs& a, int q0, int nq, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (!lattice_band_supported(a.b)) return cudaErrorInvalidValue;
    const size_t smem = window_bytes(a.b);
    if (a.b > kNarrowBand) {
        cudaError_t e = cudaFuncSetAttribute(lattice_kernel<kWideWarps>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        lattice_kernel<kWideWarps><<<nq, kWideThreads, smem, st>>>(a, q0, nq);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(lattice_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    lattice_kernel<1><<<nq, 32, smem, st>>>(a, q0, nq);
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
    const int nq = a.nspin * a.nw;
    for (int q0 = 0; q0 < nq; q0 += chunk) {
        e = launch_lattice(a, q0, std::min(chunk, nq - q0), st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hfk
