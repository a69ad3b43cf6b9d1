// k_fourier.cu -- Weiss fields and imaginary-time <-> Matsubara transforms (sm_103a, FP64).
//
// The paper keeps 500 Matsubara frequencies explicitly and solves each impurity in imaginary
// time ("Model and Methods"); the transforms themselves are not written down there.  This file
// implements the readings stated in the design notes:
//   * bath of an impurity: 1/G0 = 1/G_ii + Sigma_i (eq. 2's local self-energy), and the
//     Hartree-shifted bath of the symmetric decoupling 1/G~0 = 1/G0 - U/2;
//   * i w -> tau with the analytic tail 1/(iw) + c2/(iw)^2 + c3/(iw)^3 subtracted,
//     c2 = V_i - mu + U/2, c3 = c2^2 + z_i t^2, positive convention g(tau) = -G(tau):
//       g(tau) = -(2/beta) sum_n Re[e^{-i w_n tau}(G - tail)] + 1/2 + c2 (beta - 2 tau)/4
//                - c3 tau (beta - tau)/4;
//   * tau -> i w: G_imp(iw) = G~0(iw) + FT[-spline(g_imp - g~0)] with a natural cubic spline
//     through tau_m = m dtau, m = 0..L (g(beta-) = 1 - g(0+)), integrated exactly per segment;
//   * Sigma_new = 1/G0 - 1/G_imp, Sigma <- mix Sigma_new + (1 - mix) Sigma.
// One block per (site, spin); every loop is over at most nw = 500 frequencies or L slices.
#include "hf_internal.cuh"
#include "k_lattice.cuh"

namespace hfk {
namespace {

__device__ __forceinline__ double2 cmulf(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 crcp(double2 a) {
    const double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}

__global__ void weiss_tau_kernel(const FourierArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    double2* rem = reinterpret_cast<double2*>(smem);   // [nw]
    const int q = blockIdx.x;                          // site * 2 + spin
    const int nw = A.nw, L = A.L;
    const double beta = A.beta;
    const double c2 = A.c23[(q >> 1) * 2 + 0];
    const double c3 = A.c23[(q >> 1) * 2 + 1];
    for (int n = threadIdx.x; n < nw; n += blockDim.x) {
        const size_t idx = static_cast<size_t>(q) * nw + n;
        const double wn = (2.0 * n + 1.0) * M_PI / beta;
        const double2 wi = make_double2(crcp(A.gloc[idx]).x + A.sigma[idx].x,
                                        crcp(A.gloc[idx]).y + A.sigma[idx].y);
        A.weiss_inv[idx] = wi;
        const double2 gw = crcp(make_double2(wi.x - 0.5 * A.U, wi.y));
        A.gwt[idx] = gw;
        // tail 1/(iw) + c2/(iw)^2 + c3/(iw)^3 = (-c2/w^2) + i(-1/w + c3/w^3)
        const double tre = -c2 / (wn * wn);
        const double tim = -1.0 / wn + c3 / (wn * wn * wn);
        rem[n] = make_double2(gw.x - tre, gw.y - tim);
    }
    __syncthreads();
    for (int m = threadIdx.x; m < L; m += blockDim.x) {
        const double tau = beta * m / L;
        double s = 0.0;
        for (int n = 0; n < nw; ++n) {
            const double wn = (2.0 * n + 1.0) * M_PI / beta;
            double sn, cs;
            sincos(wn * tau, &sn, &cs);
            s += cs * rem[n].x + sn * rem[n].y;   // Re[e^{-i w tau} rem]
        }
        A.gtau[static_cast<size_t>(q) * L + m] =
            -(2.0 / beta) * s + 0.5 + c2 * (beta - 2.0 * tau) / 4.0 - c3 * tau * (beta - tau) / 4.0;
    }
}

__global__ void sigma_update_kernel(const FourierArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int L = A.L, nw = A.nw;
    double* y = reinterpret_cast<double*>(smem);   // [L+1]
    double* M2 = y + (L + 1);                      // [L+1] second derivatives
    double* cp = M2 + (L + 1);                     // [L+1] Thomas scratch
    double* co = cp + (L + 1);                     // [4L] a, b, c, d per segment
    const int q = blockIdx.x;
    const int site = q >> 1, sp = q & 1;
    const double beta = A.beta, h = beta / L;
    const double* meas = A.obs_mean + static_cast<size_t>(site) * (2 * L + 4) + sp * L;
    for (int m = threadIdx.x; m < L; m += blockDim.x)
        y[m] = meas[m] - A.gtau[static_cast<size_t>(q) * L + m];
    __syncthreads();
    if (threadIdx.x == 0) {
        y[L] = -y[0];
        // natural spline: M_0 = M_L = 0, M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1})/h^2
        M2[0] = 0.0;
        M2[L] = 0.0;
        const int n = L - 1;  // unknowns M_1..M_{L-1}
        if (n >= 1) {
            // Thomas algorithm on the constant tridiagonal (1, 4, 1) system
            double* dd = co;  // right-hand sides, reused
            for (int k = 1; k <= n; ++k) dd[k] = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) / (h * h);
            cp[1] = 1.0 / 4.0;
            dd[1] = dd[1] / 4.0;
            for (int k = 2; k <= n; ++k) {
                const double den = 4.0 - cp[k - 1];
                cp[k] = 1.0 / den;
                dd[k] = (dd[k] - dd[k - 1]) / den;
            }
            M2[n] = dd[n];
            for (int k = n - 1; k >= 1; --k) M2[k] = dd[k] - cp[k] * M2[k + 1];
        }
        for (int m = 0; m < L; ++m) {
            co[4 * m + 0] = y[m];
            co[4 * m + 1] = (y[m + 1] - y[m]) / h - h * (2.0 * M2[m] + M2[m + 1]) / 6.0;
            co[4 * m + 2] = M2[m] / 2.0;
            co[4 * m + 3] = (M2[m + 1] - M2[m]) / (6.0 * h);
        }
    }
    __syncthreads();
    for (int n = threadIdx.x; n < nw; n += blockDim.x) {
        const size_t idx = static_cast<size_t>(q) * nw + n;
        const double wn = (2.0 * n + 1.0) * M_PI / beta;
        // 1/(iw)^{k+1}, k = 0..3
        double2 ip[4];
        ip[0] = make_double2(0.0, -1.0 / wn);
        for (int k = 1; k < 4; ++k) ip[k] = cmulf(ip[k - 1], ip[0]);
        double se, ce;
        sincos(wn * h, &se, &ce);
        const double2 eh = make_double2(ce, se);
        double2 tot = make_double2(0.0, 0.0);
        for (int m = 0; m < L; ++m) {
            const double a = co[4 * m], b = co[4 * m + 1], c = co[4 * m + 2], d = co[4 * m + 3];
            const double pk_h[4] = {a + b * h + c * h * h + d * h * h * h,
                                    b + 2.0 * c * h + 3.0 * d * h * h, 2.0 * c + 6.0 * d * h,
                                    6.0 * d};
            const double pk_0[4] = {a, b, 2.0 * c, 6.0 * d};
            double2 seg = make_double2(0.0, 0.0);
            for (int k = 0; k < 4; ++k) {
                const double2 num = make_double2(eh.x * pk_h[k] - pk_0[k], eh.y * pk_h[k]);
                const double2 term = cmulf(num, ip[k]);
                const double sg = (k & 1) ? -1.0 : 1.0;
                seg.x += sg * term.x;
                seg.y += sg * term.y;
            }
            double st, ct;
            sincos(wn * (m * h), &st, &ct);
            const double2 e0 = make_double2(ct, st);
            const double2 add = cmulf(e0, seg);
            tot.x += add.x;
            tot.y += add.y;
        }
        const double2 gw = A.gwt[idx];
        const double2 gi = make_double2(gw.x - tot.x, gw.y - tot.y);
        A.gimp[idx] = gi;
        const double2 rg = crcp(gi);
        const double2 wi = A.weiss_inv[idx];
        const double2 sn = make_double2(wi.x - rg.x, wi.y - rg.y);
        A.sigma_new[idx] = sn;
        const double2 so = A.sigma[idx];
        A.sigma[idx] = make_double2(A.mix * sn.x + (1.0 - A.mix) * so.x,
                                    A.mix * sn.y + (1.0 - A.mix) * so.y);
    }
}

}  // namespace

cudaError_t launch_weiss_tau(const FourierArgs& a, cudaStream_t st) {
    if (a.nsite <= 0) return cudaSuccess;
    const size_t smem = static_cast<size_t>(a.nw) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(weiss_tau_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    weiss_tau_kernel<<<a.nsite * 2, 128, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sigma_update(const FourierArgs& a, cudaStream_t st) {
    if (a.nsite <= 0) return cudaSuccess;
    const size_t smem = static_cast<size_t>(3 * (a.L + 1) + 4 * a.L) * sizeof(double);
    sigma_update_kernel<<<a.nsite * 2, 128, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hfk
