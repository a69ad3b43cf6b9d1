// k_lattice_dev.cuh -- device helpers shared by the two lattice-step (eq. 2) kernels: complex
// FP64 arithmetic, the (w_n, sigma) item of a launch, the diagonal of M and the output of G_kk.
#pragma once

#include <cuda_runtime.h>

#include "k_lattice.cuh"

namespace hfk {

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

}  // namespace hfk
