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
// matrix; a wide one a block with two threads per window row, so that every scheduler of the SM
// has two warps issuing FP64 work (this GPU executes 2 FP64 FMA lanes per clock per SM).
#include <algorithm>
#include <atomic>

#include "hf_internal.cuh"

#include "k_lattice.cuh"
#include "k_lattice_dev.cuh"

namespace hfk {
namespace {

constexpr int kNarrowBand = 32;

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

template <bool kBlock>
__device__ __forceinline__ void mat_sync() {
    if constexpr (kBlock) __syncthreads(); else __syncwarp();
}

// Slot of index k + d given the slot sk of k (0 <= d < S).
__device__ __forceinline__ int slot(int sk, int d, int S) {
    const int v = sk + d;
    return v >= S ? v - S : v;
}

// One matrix per warp (kBlock = false; several warps, i.e. matrices, per block) or per block
// (kBlock = true; blockDim.x threads).  The selected-inversion products go a row per thread (warp
// form) or per pair of adjacent lanes (block form: two threads per window row, so two warps per
// scheduler), with no cross-lane sums on the FP64 pipe beyond one per row; the trailing update of
// the factorisation walks the triangle d2 <= d1 in one flat order shared evenly by the threads;
// the global loads of the next step (the entering row of M, the next column of L) are issued
// before the arithmetic of the current one.
template <bool kBlock>
__global__ void __launch_bounds__(384, 1) lattice_kernel(const LatticeArgs A, int q0, int nq) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = kBlock ? static_cast<int>(blockDim.x) : 32;
    const int tid = kBlock ? static_cast<int>(threadIdx.x) : static_cast<int>(threadIdx.x & 31);
    const int lane = threadIdx.x & 31;
    const int warp = tid >> 5;
    const int mi = kBlock ? 0 : static_cast<int>(threadIdx.x >> 5);
    const int qi = kBlock ? static_cast<int>(blockIdx.x)
                          : static_cast<int>(blockIdx.x * (blockDim.x >> 5)) + mi;
    if (qi >= nq) return;      // one warp of a multi-matrix block; no block barriers follow
    int sp, n;
    item_of(A, q0 + qi, sp, n);
    const int N = A.N, b = A.b, S = A.b + 1;
    const double wn = (2.0 * n + 1.0) * M_PI / A.beta;
    double2* Lg = A.scratch + static_cast<size_t>(qi) * N * S;    // Lg[k*S] = D_k, [k*S+d] = L_{k+d,k}
    double2* W = reinterpret_cast<double2*>(smem) + static_cast<size_t>(mi) * (S * (S + 1) / 2 + 3 * S);
    double2* lvb = W + S * (S + 1) / 2;   // two columns of L, [S] each (buffer p at lvb + p S)
    double2* vv = lvb + 2 * S;            // [S]
    double2* lv = lvb;
    bool bad = false;

    // 1. the window starts as the leading (b+1) x (b+1) block of M (slot = index)
    const int n0 = min(S, N);
    for (int t = tid; t < n0 * (n0 + 1) / 2; t += T) {
        int i = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while (i * (i + 1) / 2 > t) --i;
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        W[t] = m_entry(A, i, t - i * (i + 1) / 2, sp, n, wn);
    }
    mat_sync<kBlock>();

    // 2. band LDL^T, right-looking, on the window
    for (int k = 0; k < N; ++k) {
        const int dmax = min(b, N - 1 - k);
        const int sk = k % S;
        const double2 Dk = W[wtri(sk, sk)];
        const double2 inv = crecip(Dk);
        for (int d = 1 + tid; d <= dmax; d += T) {
            const double2 v = W[wtri(slot(sk, d, S), sk)];
            const double2 l = cmul(v, inv);
            vv[d] = v;
            lv[d] = l;
            Lg[static_cast<size_t>(k) * S + d] = l;
        }
        if (tid == 0) {
            Lg[static_cast<size_t>(k) * S] = Dk;
            if (!(fabs(Dk.x) + fabs(Dk.y) > 0.0) || !isfinite(Dk.x) || !isfinite(Dk.y)) bad = true;
        }
        mat_sync<kBlock>();
        // index k + b + 1 enters the slot of k (the load is issued before the update)
        const int inew = k + S;
        const int j0 = k + 1 + tid;
        const bool has_new = inew < N && j0 <= inew;
        const double2 newv = has_new ? m_entry(A, inew, j0, sp, n, wn) : make_double2(0.0, 0.0);
        // trailing update M[k+d1][k+d2] -= L_{k+d1,k} v_d2 over the flat triangle
        // f = d1 (d1 - 1) / 2 + d2 - 1 (1 <= d2 <= d1 <= dmax)
        const int E = dmax * (dmax + 1) / 2;
        if (tid < E) {
            int d1 = static_cast<int>((sqrtf(8.0f * tid + 1.0f) + 1.0f) * 0.5f);
            while (d1 * (d1 - 1) / 2 > tid) --d1;
            while (d1 * (d1 + 1) / 2 <= tid) ++d1;
            int d2 = tid - d1 * (d1 - 1) / 2 + 1;
            for (int f = tid; f < E; f += T) {
                double2* t = W + wtri(slot(sk, d1, S), slot(sk, d2, S));
                *t = cfms(*t, lv[d1], vv[d2]);
                d2 += T;
                while (d2 > d1) { d2 -= d1; ++d1; }
            }
        }
        if (has_new) W[wtri(sk, j0 % S)] = newv;
        for (int j = j0 + T; j <= inew && inew < N; j += T) W[wtri(sk, j % S)] = m_entry(A, inew, j, sp, n, wn);
        mat_sync<kBlock>();
    }

    // 3. selected inversion, k = N-1 .. 0; the window now holds Z for the indices in (k, k+b].
    // buffer k & 1 holds column k of L (entry 0: D_k), the other one receives column k - 1.
    if (tid == 0) lvb[((N - 1) & 1) * S] = Lg[static_cast<size_t>(N - 1) * S];
    mat_sync<kBlock>();
    for (int k = N - 1; k >= 0; --k) {
        const int dmax = min(b, N - 1 - k);
        const int sk = k % S;
        const double2* cur = lvb + (k & 1) * S;
        double2* nxt = lvb + ((k + 1) & 1) * S;
        const int dprev = min(b, N - k);           // dmax of step k - 1
        const bool has_pre = k > 0 && tid <= dprev;
        const double2 pre = has_pre ? Lg[static_cast<size_t>(k - 1) * S + tid] : make_double2(0.0, 0.0);
        // Z_{k+d,k} = -sum_e Z_{k+d,k+e} L_{k+e,k}: a row per thread (warp form) or per pair of
        // adjacent lanes, each summing alternate e (block form: two warps per scheduler)
        if constexpr (kBlock) {
            // rows r0 + lane / 2 of this warp; the loop bound is uniform over the warp, so every
            // lane reaches the pair shuffle (lanes past dmax contribute nothing)
            const int h = lane & 1;
            for (int r0 = (tid - lane) >> 1; r0 < dmax; r0 += (T >> 1)) {
                const int d = r0 + (lane >> 1) + 1;
                double2 a0 = make_double2(0.0, 0.0), a1 = a0;
                if (d <= dmax) {
                    const int s1 = slot(sk, d, S);
                    int e = 1 + h;
                    for (; e + 2 <= dmax; e += 4) {
                        a0 = cfms(a0, W[wtri(s1, slot(sk, e, S))], cur[e]);
                        a1 = cfms(a1, W[wtri(s1, slot(sk, e + 2, S))], cur[e + 2]);
                    }
                    if (e <= dmax) a0 = cfms(a0, W[wtri(s1, slot(sk, e, S))], cur[e]);
                }
                const double2 a = make_double2(a0.x + a1.x, a0.y + a1.y);
                const double2 o = shfl_xor_c(a, 1);
                if (h == 0 && d <= dmax) vv[d] = make_double2(a.x + o.x, a.y + o.y);
            }
        } else {
            for (int d = 1 + tid; d <= dmax; d += T) {
                const int s1 = slot(sk, d, S);
                double2 a0 = make_double2(0.0, 0.0), a1 = a0;
                int e = 1;
                for (; e + 1 <= dmax; e += 2) {
                    a0 = cfms(a0, W[wtri(s1, slot(sk, e, S))], cur[e]);
                    a1 = cfms(a1, W[wtri(s1, slot(sk, e + 1, S))], cur[e + 1]);
                }
                if (e <= dmax) a0 = cfms(a0, W[wtri(s1, slot(sk, e, S))], cur[e]);
                vv[d] = make_double2(a0.x + a1.x, a0.y + a1.y);
            }
        }
        mat_sync<kBlock>();
        // row/column k into the slot of k (which held k + b + 1, outside every later window)
        for (int d = 1 + tid; d <= dmax; d += T) W[wtri(sk, slot(sk, d, S))] = vv[d];
        if (warp == 0) {
            double2 part = make_double2(0.0, 0.0);
            for (int d = 1 + lane; d <= dmax; d += 32) part = cfms(part, cur[d], vv[d]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double2 t = shfl_xor_c(part, o);
                part.x += t.x;
                part.y += t.y;
            }
            if (lane == 0) {
                const double2 ri = crecip(cur[0]);
                const double2 zkk = make_double2(ri.x + part.x, ri.y + part.y);
                W[wtri(sk, sk)] = zkk;
                store_diag(A, k, sp, n, zkk);
                if (!isfinite(zkk.x) || !isfinite(zkk.y)) bad = true;
            }
        }
        if (has_pre) nxt[tid] = pre;
        if (k > 0)
            for (int e = tid + T; e <= dprev; e += T) nxt[e] = Lg[static_cast<size_t>(k - 1) * S + e];
        mat_sync<kBlock>();
    }
    if (bad) atomicExch(A.status, static_cast<int>(HF_ENUMERIC));
}

size_t window_bytes(int b) {     // one matrix: packed window and three vectors
    const size_t S = static_cast<size_t>(b) + 1;
    return (S * (S + 1) / 2 + 3 * S) * sizeof(double2);
}

int block_threads(int b) {       // two threads per row of the window
    return 64 * ((b + 31) / 32);
}

}  // namespace

bool lattice_window_supported(int b) {
    return b >= 0 && window_bytes(b) <= static_cast<size_t>(227) * 1024;
}

int lattice_window_max_band() {
    int b = 0;
    while (lattice_window_supported(b + 1)) ++b;
    return b;
}

bool lattice_band_supported(int b) { return b >= 0 && b <= lattice_max_band(); }

int lattice_max_band() { return std::max(lattice_window_max_band(), lattice_wide_max_band()); }

size_t lattice_scratch_per_matrix(int N, int b) {
    return static_cast<size_t>(N) * (b + 1) * sizeof(double2);
}

cudaError_t launch_lattice(const LatticeArgs& a, int q0, int nq, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (a.wide || !lattice_window_supported(a.b)) return launch_lattice_wide(a, q0, nq, st);
    const size_t smem = window_bytes(a.b);
    if (a.b > kNarrowBand) {
        cudaError_t e = cudaFuncSetAttribute(lattice_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        lattice_kernel<true><<<nq, block_threads(a.b), smem, st>>>(a, q0, nq);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(lattice_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    lattice_kernel<false><<<nq, 32, smem, st>>>(a, q0, nq);
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

// task counter and ready flags of the blocked band form, for chunks of up to kStaticChunk matrices
constexpr int kStaticChunk = 4096;
static __device__ int g_lattice_work[kStaticChunk + 1];

size_t lattice_static_scratch_bytes() { return kStaticLatticeScratchBytes; }

// Device addresses of g_lattice_scratch and g_lattice_work on the current device, looked up
// once per device (the host-side symbols are only stand-ins and must never reach a kernel).  The
// per-device entries are atomics: host threads that make their first call on a device at the
// same time each look the addresses up and store the same values.
static cudaError_t static_scratch_address(double2** out, int** work) {
    constexpr int kMaxDevices = 64;
    static std::atomic<double2*> addr[kMaxDevices] = {};
    static std::atomic<int*> waddr[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    double2* a = addr[dev].load(std::memory_order_acquire);
    int* w = waddr[dev].load(std::memory_order_acquire);
    if (a == nullptr || w == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_lattice_scratch);
        if (e != cudaSuccess) return e;
        a = static_cast<double2*>(p);
        e = cudaGetSymbolAddress(&p, g_lattice_work);
        if (e != cudaSuccess) return e;
        w = static_cast<int*>(p);
        addr[dev].store(a, std::memory_order_release);
        waddr[dev].store(w, std::memory_order_release);
    }
    *out = a;
    *work = w;
    return cudaSuccess;
}

cudaError_t launch_lattice_static(const LatticeArgs& a_in, cudaStream_t st) {
    const size_t per = lattice_scratch_per_matrix(a_in.N, a_in.b);
    if (per == 0 || per > kStaticLatticeScratchBytes) return cudaErrorInvalidValue;
    double2* base = nullptr;
    int* work = nullptr;
    cudaError_t e = static_scratch_address(&base, &work);
    if (e != cudaSuccess) return e;
    LatticeArgs a = a_in;
    a.scratch = base;
    a.work = work;
    const int chunk = static_cast<int>(std::min<size_t>(kStaticChunk, kStaticLatticeScratchBytes / per));
    const int nq = a.nspin * a.nw;
    for (int q0 = 0; q0 < nq; q0 += chunk) {
        e = launch_lattice(a, q0, std::min(chunk, nq - q0), st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hfk
