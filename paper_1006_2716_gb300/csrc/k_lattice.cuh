// k_lattice.cuh -- arguments of the lattice-step (eq. 2) and transform kernels.
#pragma once

#include <cuda_runtime.h>

namespace hfk {

struct LatticeArgs {
    int N, b, nw;             // lattice sites, band half-width, Matsubara frequencies
    double beta, mu;
    const double* h0band;     // [N][b+1]: H0[k+d][k] (d = 0: trap potential V_k)
    const int* rep_of;        // [N] inequivalent index of each site
    const int* flip;          // [N] 1: spins exchanged relative to the representative
    const int* site_rep;      // [N] inequivalent index if the site is a representative, else -1
    const int* site_dn;       // [N] or nullptr: inequivalent index r whose spin-down G_rr equals
                              //     the spin-up G at this position, else -1 (nspin = 1)
    int nspin;                // 2: a matrix per (w_n, sigma); 1: spin-up matrices only
    const double2* sigma;     // [nsite][2][nw]
    double2* gloc;            // [nsite][2][nw] output G_ii of the representatives
    double2* scratch;         // [nq][N][b+1] band factors of the matrices in flight (q = sigma nw + n)
    int* status;
    // blocked band form (k_lattice_wide.cu): G_kk only at listed band positions, one per output
    int wide;                 // 1: blocked band form for this lattice (always above the window)
    int wide_npos;            // listed positions per spin matrix
    const int* wide_pos;      // [nspin][wide_npos] band positions to solve for, ascending
    const int* wide_out;      // [nspin][wide_npos] row r * 2 + slot of gloc that each one fills
    int* work;                // [1 + matrices per launch] task counter and per-matrix ready flags
};

// Shared-memory window form (k_lattice.cu): a (b+1)(b+2)/2-entry window per matrix.
bool lattice_window_supported(int b);
int lattice_window_max_band();
// Either form: the window form up to its largest band unless a.wide, the blocked band form above.
bool lattice_band_supported(int b);
int lattice_max_band();
size_t lattice_scratch_per_matrix(int N, int b);
cudaError_t launch_lattice(const LatticeArgs& a, int q0, int nq, cudaStream_t st);

// Blocked band form (k_lattice_wide.cu), every b <= lattice_wide_max_band().
int lattice_wide_max_band();
// Smallest band half-width whose products the blocked form runs on the tensor cores.
int lattice_wide_tc_min_band();
int lattice_wide_rhs_per_block();
// bf16 flops of the tensor-core trailing updates per matrix (0 where the band keeps DFMA)
double lattice_wide_tc_flops(int N, int b, const int* pos, int npos, int nspin);
cudaError_t launch_lattice_wide(const LatticeArgs& a, int q0, int nq, cudaStream_t st);

// Lattice step over all nspin * nw matrices with the band buffers in a fixed 16 MiB device array
// (a.scratch is ignored); rejects a lattice whose single band does not fit.
size_t lattice_static_scratch_bytes();
cudaError_t launch_lattice_static(const LatticeArgs& a, cudaStream_t st);

struct FourierArgs {
    int nsite, L, nw;
    double beta, U, mix;
    const double* c23;        // [nsite][2]: tail coefficients c2, c3 of the shifted bath
    const double2* gloc;      // [nsite][2][nw]
    double2* sigma;           // [nsite][2][nw] (read, then mixed in place)
    double2* weiss_inv;       // [nsite][2][nw]  1/G0 = 1/G_ii + Sigma
    double2* gwt;             // [nsite][2][nw]  G~0 = 1/(1/G0 - U/2)
    double* gtau;             // [nsite][2][L]   g~0(tau_m)
    const double* obs_mean;   // [nsite][2L+4]   measured G(tau_m) (first 2L entries)
    double2* gimp;            // [nsite][2][nw]  impurity G(i w_n)
    double2* sigma_new;       // [nsite][2][nw]  unmixed 1/G0 - 1/G_imp
};

cudaError_t launch_weiss_tau(const FourierArgs& a, cudaStream_t st);
cudaError_t launch_sigma_update(const FourierArgs& a, cudaStream_t st);

}  // namespace hfk
