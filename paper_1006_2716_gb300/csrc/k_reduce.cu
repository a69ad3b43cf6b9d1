// k_reduce.cu -- chain x bin reduction of the QMC measurements (sm_103a).
//
// Per inequivalent site: mean and standard error over (chain, bin) of the bin averages of
// G_up(tau_m), G_dn(tau_m), n_up, n_dn, double occupancy and m = n_up - n_dn.  Bins are
// treated as independent samples (bin size chosen well above the autocorrelation time).
#include "hf_internal.cuh"

namespace hfk {
namespace {

__global__ void reduce_kernel(const double* __restrict__ bins, int cps, int L, int max_bins,
                              int nb, int bin_size, double* __restrict__ mean,
                              double* __restrict__ err) {
    const int site = blockIdx.x;
    const int W = 2 * L + 3;
    const int K = 2 * L + 4;
    const double inv_bs = 1.0 / bin_size;
    const long n = static_cast<long>(cps) * nb;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double sum = 0.0;
        for (int c = 0; c < cps; ++c) {
            const double* bc = bins + (static_cast<size_t>(site) * cps + c) * max_bins * W;
            for (int b = 0; b < nb; ++b) {
                const double* x = bc + static_cast<size_t>(b) * W;
                const double v = (k < W) ? x[k] : (x[2 * L] - x[2 * L + 1]);
                sum += v * inv_bs;
            }
        }
        const double mu = (n > 0) ? sum / static_cast<double>(n) : 0.0;
        double ss = 0.0;
        for (int c = 0; c < cps; ++c) {
            const double* bc = bins + (static_cast<size_t>(site) * cps + c) * max_bins * W;
            for (int b = 0; b < nb; ++b) {
                const double* x = bc + static_cast<size_t>(b) * W;
                const double v = ((k < W) ? x[k] : (x[2 * L] - x[2 * L + 1])) * inv_bs - mu;
                ss += v * v;
            }
        }
        mean[static_cast<size_t>(site) * K + k] = mu;
        err[static_cast<size_t>(site) * K + k] =
            (n > 1) ? sqrt(ss / static_cast<double>(n - 1) / static_cast<double>(n)) : 0.0;
    }
}

}  // namespace

cudaError_t launch_reduce(const double* bins, int nsite, int cps, int L, int max_bins,
                          int nbins_done, int bin_size, double* out_mean, double* out_err,
                          cudaStream_t st) {
    if (nsite <= 0) return cudaSuccess;
    reduce_kernel<<<nsite, 128, 0, st>>>(bins, cps, L, max_bins, nbins_done, bin_size,
                                         out_mean, out_err);
    return cudaGetLastError();
}

}  // namespace hfk
