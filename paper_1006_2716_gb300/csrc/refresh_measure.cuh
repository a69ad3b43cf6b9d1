// refresh_measure.cuh -- the measurement that follows an FP64 refresh of the mixed-precision form:
// G(tau_m), n_sigma and the double occupancy of one chain, from the FP64 G the refresh wrote,
// added to the chain's current bin.
#pragma once

#include "hf_internal.cuh"

namespace hfk {

// One CTA of NT threads (a multiple of 32, at most 1024) measures chain c (P.L slices); red is
// shared scratch of at least 3 NT / 32 doubles.  Reads the chain's FP64 G (written by this CTA before a
// __syncthreads).
template <int NT>
__device__ void measure_refreshed(const QmcProblem& P, int c, double* red) {
    const int L = P.L;
    const int LL = L * L;
    const int tid = threadIdx.x;
    const int W = 2 * L + 3;
    const uint32_t nmeas = P.nmeas[c];
    const int b = static_cast<int>(nmeas / P.bin_size);
    double* bin = P.bins + (static_cast<size_t>(c) * P.max_bins + b) * W;
    const double* G0 = P.G + static_cast<size_t>(c) * 2 * LL;
    const double* G1 = G0 + LL;
    // G(tau_m) = (1/L) sum_l sgn G[(l+m) mod L][l] (sgn = -1 on wrap); thread m walks l in a
    // skewed order so that the lanes of a warp read different rows
    for (int m = tid; m < L; m += NT) {
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
    for (int l = tid; l < L; l += NT) {
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
    constexpr int NW = NT / 32;
    const int w = tid >> 5;
    if ((tid & 31) == 0) {
        red[w] = nu;
        red[NW + w] = nd;
        red[2 * NW + w] = db;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, bb = 0.0, cc = 0.0;
        for (int k = 0; k < NW; ++k) {
            a += red[k];
            bb += red[NW + k];
            cc += red[2 * NW + k];
        }
        if (b < P.max_bins) {
            bin[2 * L + 0] += a / L;
            bin[2 * L + 1] += bb / L;
            bin[2 * L + 2] += cc / L;
        }
        P.nmeas[c] = nmeas + 1;
    }
}

}  // namespace hfk
