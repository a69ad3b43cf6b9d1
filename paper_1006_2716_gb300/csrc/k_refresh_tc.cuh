// k_refresh_tc.cuh -- the tensor-core FP64 Dyson refresh of the mixed-precision form (L = 128)
// and the FP64-accurate 128 x 128 product it is built from.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hf_internal.cuh"

namespace hfk {

constexpr int kTcL = 128;              // the slice count the tensor-core refresh handles
constexpr int kTcDigits = 8;           // balanced base-256 digits kept of an operand at most

// Extra device buffers of the tensor-core refresh of one problem (all in the context workspace).
struct TcRefreshArgs {
    uint16_t* g0inv_digits;   // [nsite][2][kTcDigits][128*128] bf16 digits of g0^{-1}, chunked
    int* g0inv_rowT;          // [nsite][2][128] power-of-two row scales of g0^{-1}
    double* scratch;          // [nchain][128*128] FP64 residual / iterate buffer
    int* fail;                // [nchain] 1 = the chain needs the Gauss-Jordan refresh
    int* fail_list;           // [nchain] the chains with fail set, in no particular order
    int* fail_count;          // [1] entries of fail_list (cleared before each refresh launch)
    unsigned long long* products;  // [1] 128 x 128 x 128 digit products run (bf16 MMA work)
};

size_t tc_digits_bytes(int nsite);        // bytes of g0inv_digits
size_t tc_refresh_smem_bytes();

// Digits and row scales of every site's g0^{-1} (after launch_g0_inverse, whenever a bath
// changes).
cudaError_t launch_g0inv_digits(const QmcProblem& p, const TcRefreshArgs& a, cudaStream_t st);

// Refresh of every chain of p (L = 128): G = M^{-1}, M = g0^{-1} e^V - (e^V - 1), by two Newton
// steps X <- X + X (1 - M X) from the chain's FP32 state, the residual products formed exactly
// on the tensor cores; writes the FP64 G and its FP32 copy and, with p.refresh_measure, the
// measurement.  A chain whose residual does not fall below the convergence bound (or whose
// scales leave the fixed-point range) is left untouched, with a.fail set and its index appended
// to a.fail_list; launch_refresh_f64_listed then refreshes it by Gauss-Jordan elimination.  The
// caller clears *a.fail_count before the launch.
cudaError_t launch_refresh_tc(const QmcProblem& p, const TcRefreshArgs& a, cudaStream_t st);

// The Gauss-Jordan FP64 refresh of the chains listed in list[0 .. *count) (k_qmc_f32.cu): one
// wave of CTAs that take the listed chains in turn, so an empty list costs one short launch.
cudaError_t launch_refresh_f64_listed(const QmcProblem& p, const int* list, const int* count,
                                      cudaStream_t st);

// C_b = A_b B_b for n pairs of row-major 128 x 128 FP64 matrices, each operand cut into
// `digits` balanced base-256 digits (1, 3, 5, 7 or 8) and the levels s + t <= digits + 1 formed
// on the tensor cores.
cudaError_t launch_tc_dgemm128(const double* A, const double* B, double* C, int n, int digits,
                               int* status, cudaStream_t st);

}  // namespace hfk
