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
// every diagonal element.  For 128 <= b <= kTcMaxBand the products (a panel's rows below its
// diagonal block, the trailing updates, the solves' row updates) run on the tensor cores as
// exact digit products, each entry rounded once to FP64; the rest stays on the FP64 pipe.
#include <algorithm>

#include "hf_internal.cuh"

#include "k_lattice.cuh"
#include "k_lattice_dev.cuh"
#include "tc_ozaki.cuh"

namespace hfk {
namespace {

constexpr int kNB = 16;          // panel width
constexpr int kT = 512;          // threads of a block (both kinds of task)
constexpr int kR = 16;           // right-hand sides per solve task
constexpr int kWideMaxBand = 840;
constexpr int kSeg = 256;        // rows of a trailing-update unit (8 per lane)

static_assert(kWideMaxBand <= 2 * kT, "two band entries of a column per solve thread at most");

// Row stride of the staged panel: kNB + b rows, rounded up to an odd count so that the 16
// columns of one row fall in different shared-memory banks.
__host__ __device__ constexpr int panel_stride(int b) { return (kNB + b) | 1; }

size_t factor_smem(int b) {      // the panel and the pivot row
    return (static_cast<size_t>(kNB) * panel_stride(b) + kNB) * sizeof(double2);
}

size_t solve_smem(int b) {       // kR windows of b + 1 entries
    return static_cast<size_t>(kR) * (b + 1) * sizeof(double2);
}

// ---- the products on the tensor cores (128 <= b <= kTcMaxBand) ----
// The trailing update A[r][c] -= sum_j L_rj W_cj, W_cj = D_j L_cj, the panel's rows below its
// diagonal block and the forward solves' updates run as exact digit products (the error-free
// splitting of tc_ozaki.cuh).  For the trailing update, with A = [Re W | Im W] (128 trailing
// columns c per tile, K = 32: the panel's 16 columns, real and imaginary parts) and
// B_re = [Re L | -Im L], B_im = [Im L | Re L] (16 trailing rows r per tile), Re and Im of the
// sum are A B_re^T and A B_im^T.  Each operand row gets a power-of-two scale and kTD balanced
// base-256 digits; the levels n = s + t <= kTNL are kept (the dropped ones stay below 2^-58 of
// the scales), each an exact FP32 accumulator in TMEM (K = 32 terms of at most 2^14, at most 7
// per level: below 2^22).  A digit plane of B holds the B_re and B_im rows of the tile's 16
// rows r, interleaved by eights (row 16 (r / 8) + 8 part + r % 8), so a level's accumulator is
// 32 TMEM columns in which each thread's 8 rows r have their Re and Im sums side by side; eight
// levels take 256 columns, half of TMEM.  For each digit s of A the digits t of B are stacked
// along N (up to eight planes, 256 columns, per MMA): 15 MMAs per tile, each reading its A plane
// once for up to 256 columns.  The epilogue combines a tile's levels in 64-bit integers and
// subtracts the rounded sums from the band buffer in FP64: one DADD per part and entry per
// panel, against 16 complex multiply-adds.
constexpr int kTD = 7;                  // digits of an operand
constexpr int kTNL = kTD + 2;           // highest level kept
static_assert((kTNL - 1) % 2 == 0, "the levels 2 .. kTNL pair up");
constexpr int kTM = 128;                // rows of A per tile (MMA M): trailing columns c, rows
constexpr int kTK = 32;                 // K
constexpr int kPlaneA = kTM * kTK * 2;  // bytes of one digit plane of A (K-major core matrices)
constexpr int kTcMinBand = 128;
constexpr int kTcMaxBand = 520;
// Every product has 16 complex columns on the B side (16 trailing rows, the panel's 16 columns
// of Z, 16 right-hand sides): a digit plane of B holds their Re and Im rows, 32 rows of K = 32.
constexpr int kSN = 16;
constexpr int kPlaneS = 2 * kSN * kTK * 2;
static_assert(kSN == kR, "a solve task's right-hand sides fill the B side");

struct TcSmem {                         // behind the panel, 1024-byte aligned
    unsigned char a[kTD * kPlaneA];
    unsigned char b[2 * kTD * kPlaneS];  // B planes: one set per warp group (trailing update)
    int ta[kTM];                        // scales of A's rows (the tile's columns c)
    int tb[kNB + kTcMaxBand];           // scales of the B rows: the panel's rows (trailing
                                        // update), the right-hand sides (solve)
    uint64_t bar[4];                    // MMA completion (the trailing update's warp groups;
                                        // the panels and solves use bar[0])
    uint32_t tmem;                      // TMEM base address
    int fail;                           // an MMA wait ran out: no more tensor-core work
};

size_t tc_offset(int b) { return (factor_smem(b) + 1023) / 1024 * 1024; }
__device__ __forceinline__ int tc_offset_dev(int b) {
    return ((kNB * panel_stride(b) + kNB) * static_cast<int>(sizeof(double2)) + 1023) / 1024 * 1024;
}

size_t wide_smem(int b, bool tc) {
    const size_t f = tc ? tc_offset(b) + sizeof(TcSmem) : factor_smem(b);
    return std::max(f, solve_smem(b));
}

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

// kTD balanced base-256 digits of 4 fixed-point magnitudes (top down, each rounded) into the
// digit planes at base (plane stride `plane`), 8 bytes at offset off of each.
__device__ __forceinline__ void put_digits4(const unsigned long long (&U)[4], const bool (&neg)[4],
                                            unsigned char* base, int plane, int off) {
    long long r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = static_cast<long long>(U[q]);
#pragma unroll
    for (int sd = 1; sd <= kTD; ++sd) {
        const int sh = 62 - 8 * sd;
        int d[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long v = (r[q] + (1ll << (sh - 1))) >> sh;
            r[q] -= v << sh;
            d[q] = static_cast<int>(v);
        }
        *reinterpret_cast<uint2*>(base + (sd - 1) * plane + off) =
            make_uint2(tc::bf16x2_digits(d[0], d[1], neg[0], neg[1]), tc::bf16x2_digits(d[2], d[3], neg[2], neg[3]));
    }
}

// Digit-plane offset of element (row m, k) of a K-major operand with K = 32: 8-row x 16-byte
// core matrices, 128 bytes apart along K, 512 bytes apart along the rows.
__device__ __forceinline__ int core_off(int m, int kg) { return ((m >> 3) * 4 + kg) * 128 + (m & 7) * 16; }

__device__ __forceinline__ int scale_of(int e) { return e == tc::kNoExp ? 0 : e + 2; }

// A level accumulator of these products (an integer below 2^22 in magnitude: K = 32 terms of at
// most 2^14, at most 7 digit pairs) as an int: adding 1.5 2^23 moves it, exactly, into the low
// bits of the significand.
__device__ __forceinline__ int level_int(uint32_t bits) {
    return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

// Adds the levels n and n + 1 (n even), combined exactly in 32 bits as d_n 2^8 + d_{n+1}
// (below 2^31), to a 64-bit sum in units of 2^-54 of the scales (rounded where the pair's
// weight 2^(54 - 8 (n + 1)) is below one unit).
__device__ __forceinline__ void add_level_pair(long long& Q, int dn, int dn1, int n) {
    const long long p = static_cast<long long>(dn * 256 + dn1);
    const int sh = 54 - 8 * (n + 1);
    Q += sh >= 0 ? (p << sh) : ((p + (1ll << (-sh - 1))) >> (-sh));
}

// The sign-flipped bit pattern of x (no FP64 instruction).
__device__ __forceinline__ double neg_bits(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ static_cast<long long>(0x8000000000000000ull));
}

// Level n of a product lives in TMEM columns W (n - 2) ... (W per level).  The digit products of
// one tile: for each digit s of A (planes (s - 1) planeA) the digits t = 1 .. min(kTD, kTNL - s)
// of B (planes (t - 1) planeB, W rows each) in runs of at most 256 / W planes, one MMA per run and
// K half, writing the level blocks s + t .. in one go.  The first product of each level
// (s = max(1, n - kTD), first K half) starts its accumulator: a run never mixes first products
// with later ones.  The schedule is fixed at compile time.
struct MmaRun {
    int kk, sd, t, nt;
    bool first;
};
template <int G>
struct MmaSchedule {
    MmaRun run[32];
    int n;
};
template <int G>
__host__ __device__ constexpr MmaSchedule<G> mma_schedule() {
    MmaSchedule<G> S{};
    for (int kk = 0; kk < 2; ++kk)
        for (int sd = 1; sd <= kTD; ++sd) {
            const int tmax = kTD < kTNL - sd ? kTD : kTNL - sd;
            int t = 1;
            while (t <= tmax) {
                const auto first_of = [&](int tt) { return kk == 0 && sd == (sd + tt - kTD > 1 ? sd + tt - kTD : 1); };
                const bool first = first_of(t);
                int e = t;
                while (e < tmax && e - t + 1 < G && first_of(e + 1) == first) ++e;
                S.run[S.n++] = MmaRun{kk, sd, t, e - t + 1, first};
                t = e + 1;
            }
        }
    return S;
}

// Issued by one thread.  adesc / bdesc: descriptors of the first A and B planes (K-major, core
// matrices 128 bytes apart along K and 512 along the rows); an offset of o bytes adds o / 16.
template <int W, int PlaneA, int PlaneB>
__device__ __forceinline__ void issue_levels(uint32_t tmem, uint64_t adesc, uint64_t bdesc) {
    constexpr MmaSchedule<256 / W> S = mma_schedule<256 / W>();
    static_assert(S.n <= 32, "schedule fits");
#pragma unroll
    for (int i = 0; i < S.n; ++i) {
        const MmaRun r = S.run[i];
        tc::mma_bf16(tmem + (r.sd + r.t - 2) * W, adesc + (((r.sd - 1) * PlaneA + r.kk * 256) >> 4),
                     bdesc + (((r.t - 1) * PlaneB + r.kk * 256) >> 4), tc::idesc_bf16_f32(kTM, r.nt * W),
                     !r.first);
    }
}

// Named barrier `id` over the `count` threads of a warp group.
__device__ __forceinline__ void group_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// The trailing update of one panel on the tensor cores: rows and columns nb .. tend of the panel
// P (RP the row stride, L_ij scaled, D_j on the diagonal) into the band buffer Bq at k0.
// Per column tile of 128 all 512 threads cut the A digits; its row tiles of kRT = 8 rows go in
// turn to the kGroups = 4 warp groups (128 threads each), each with its own B planes, its own
// quarter of TMEM (eight levels x 16 columns), its own mbarrier and a named barrier, so that one
// group's epilogue runs while the others cut digits and wait for their MMAs.  ph: bit g the phase
// of mbarrier g, flipped by every tile of group g (in every thread).
constexpr int kGroups = 4;
constexpr int kGT = kT / kGroups;                // threads of a group
constexpr int kRT = 32 / kGroups;                // trailing rows r per tile: 8 entries a thread
constexpr int kPlaneT = 2 * kRT * kTK * 2;       // one B digit plane of a trailing tile
static_assert(kRT % 8 == 0 && kGT == 16 * kRT, "a group cuts a tile's B digits, 4 K a thread");
static_assert(kGroups * kTD * kPlaneT <= 2 * kTD * kPlaneS, "the groups' B planes fit");

__device__ void trailing_tc(TcSmem& T, const double2* P, int RP, int nb, int tend, double2* Bq,
                            int k0, int S, uint32_t& ph) {
    const int tid = static_cast<int>(threadIdx.x), lane = tid & 31, warp = tid >> 5;
    const int grp = tid / kGT, u = tid % kGT;     // warp group, thread within it
    const int rows = tend - nb + 1;
    if (rows <= 0) return;
    // the B scales of every trailing row, once for the panel (a thread per row)
    for (int i = nb + tid; i <= tend; i += kT) {
        int e = tc::kNoExp;
#pragma unroll
        for (int j = 0; j < kNB; ++j) {
            const double2 l = P[j * RP + i];
            e = max(e, max(tc::exp_of(l.x), tc::exp_of(l.y)));
        }
        T.tb[i] = scale_of(e);
    }
    unsigned char* bplanes = T.b + grp * (kTD * kPlaneT);
    const uint32_t tmem = T.tmem + (512 / kGroups) * grp;
    for (int c0 = 0; c0 < rows; c0 += kTM) {
        // A: W_cj = D_j L_cj of the tile's columns c = nb + c0 + m, m < 128 (zero past tend):
        // four threads per column (adjacent lanes, four j each) form their W once, agree on the
        // column's scale by shuffle and cut the Re and Im digits
        {
            const int m = tid >> 2, part = tid & 3;
            const int c = nb + c0 + m;
            double2 w[4];
            int e = tc::kNoExp;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * part + q;
                w[q] = c <= tend ? cmul(P[j * RP + j], P[j * RP + c]) : make_double2(0.0, 0.0);
                e = max(e, max(tc::exp_of(w[q].x), tc::exp_of(w[q].y)));
            }
            e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
            e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
            const int Ta = scale_of(e);
            if (part == 0) T.ta[m] = Ta;
            unsigned long long U[4];
            bool neg[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) U[q] = tc::to_fixed_mag(w[q].x, Ta, neg[q]);
            put_digits4(U, neg, T.a, kPlaneA, core_off(m, part >> 1) + (part & 1) * 8);
#pragma unroll
            for (int q = 0; q < 4; ++q) U[q] = tc::to_fixed_mag(w[q].y, Ta, neg[q]);
            put_digits4(U, neg, T.a, kPlaneA, core_off(m, 2 + (part >> 1)) + (part & 1) * 8);
        }
        tc::fence_async_shared();
        __syncthreads();   // the A planes and scales (and, first time round, the B scales)
        const int nt = (rows - c0 + kRT - 1) / kRT;
        for (int t = 0; t < nt; ++t) {
            const int g = t % kGroups;
            if (g != grp) {            // another group's tile: only its phase bit
                ph ^= 1u << g;
                continue;
            }
            const int r0 = c0 + t * kRT;
            // B: L_rj of the tile's rows r = nb + r0 + nr, nr < kRT, as [Re | -Im] (part 0) and
            // [Im | Re] (part 1), 4 K a thread; plane row 16 (nr / 8) + 8 part + nr % 8
            {
                const int part = u / (8 * kRT), nr = u % kRT, kq = (u / kRT) % 8, kg = kq >> 1;
                const int r = nb + r0 + nr;
                const int Tb = r <= tend ? T.tb[r] : 0;
                unsigned long long U[4];
                bool neg[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = ((4 * kq + q) & 15);
                    const double2 l = r <= tend ? P[j * RP + r] : make_double2(0.0, 0.0);
                    double x;
                    if (part == 0) x = kg < 2 ? l.x : neg_bits(l.y);
                    else x = kg < 2 ? l.y : l.x;
                    U[q] = tc::to_fixed_mag(x, Tb, neg[q]);
                }
                const int mb = 16 * (nr >> 3) + 8 * part + (nr & 7);
                put_digits4(U, neg, bplanes, kPlaneT, core_off(mb, kg) + (kq & 1) * 8);
            }
            tc::fence_async_shared();
            tc::tc_fence_before_sync();
            group_sync(1 + grp, kGT);
            // the MMAs, issued by the group's first thread and committed to its mbarrier
            if (u == 0 && !T.fail) {
                tc::tc_fence_after_sync();
                issue_levels<2 * kRT, kPlaneA, kPlaneT>(tmem, tc::smem_desc(tc::smem_addr(T.a), 128, 512),
                                                        tc::smem_desc(tc::smem_addr(bplanes), 128, 512));
                tc::mma_commit(&T.bar[grp]);
            }
            // the band entries this thread updates, loaded while the MMAs run: lane quarter
            // (warp & 3) holds columns c = c0 + 32 (warp & 3) + lane, the group's warps of a
            // quarter 8 rows each (contiguous in column c); loaded unconditionally (entries
            // outside the triangle clamped onto it, their values unused)
            const int ql = warp & 3, h = (u >> 7);
            const int m = 32 * ql + lane;
            const int c = nb + c0 + m;
            const int rlo = nb + r0 + 8 * h;
            double2* col = Bq + (static_cast<size_t>(k0 + c) * S - c);   // col[r] = A[r][c]
            const int cc = min(c, tend);
            const double2* colc = Bq + (static_cast<size_t>(k0 + cc) * S - cc);
            double2 x[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = colc[min(max(rlo + k, cc), tend)];
            // wait for the group's MMAs (bounded; a wait that runs out stops the tensor-core
            // work of this block, the launch reports HF_ETIMEOUT)
            if (!T.fail && !tc::mbar_wait(&T.bar[grp], (ph >> grp) & 1u)) T.fail = 1;
            ph ^= 1u << grp;
            tc::tc_fence_after_sync();
            // epilogue: the level sums of this thread's 8 rows (Re and Im side by side)
            {
                const uint32_t trow = tmem + (static_cast<uint32_t>(32 * ql) << 16) + 16 * h;
                long long Qr[8], Qi[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) Qr[k] = Qi[k] = 0;
#pragma unroll
                for (int n = 2; n <= kTNL; n += 2)
#pragma unroll
                    for (int part = 0; part < 2; ++part) {   // Re, then Im, of the levels n, n + 1
                        uint32_t v0[8], v1[8];
                        tc::tmem_ld8_async(trow + (n - 2) * (2 * kRT) + 8 * part, v0);
                        tc::tmem_ld8_async(trow + (n - 1) * (2 * kRT) + 8 * part, v1);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            add_level_pair(part == 0 ? Qr[k] : Qi[k], level_int(v0[k]), level_int(v1[k]), n);
                    }
                if (c <= tend) {
                    const int Ta = T.ta[m];
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int r = rlo + k;
                        if (r >= c && r <= tend) {
                            const int E = Ta + T.tb[r] - 54;
                            col[r] = make_double2(x[k].x - tc::fixed_to_double(Qr[k], E),
                                                  x[k].y - tc::fixed_to_double(Qi[k], E));
                        }
                    }
                }
            }
            tc::tc_fence_before_sync();
            group_sync(1 + grp, kGT);   // the group's TMEM share and B planes are reused
        }
        __syncthreads();                // the A planes are reused by the next column tile
    }
}

// The panel of a full step with the tensor cores.  (1) Its 16 x 16 diagonal block is factored in
// FP64, a thread per pair (jp, i) of the block's lower triangle in order of falling jp, so that
// the pairs a step updates are packed into the fewest warps; the thread of the next pivot also
// forms its reciprocal, and column j - 1 is scaled during step j.  (2) X = L11^{-1} by forward
// substitution, a half warp per column of X (X[k][m] passed by shuffle).  (3) The rows below,
// L21 = A21 (D L11^T)^{-1} = A21 Z with Z[m][c] = X[c][m] / D_c, as exact digit products with
// A = [Re A21 | Im A21] (128 rows per tile) and B = [Re Z | -Im Z], [Im Z | Re Z] (the solves'
// layout), each entry rounded once.  P: the staged panel (row stride RP, rmax rows); on return
// it holds D on the diagonal and L below.  Returns false if an MMA wait ran out.
__device__ bool panel_tc(TcSmem& T, double2* P, int RP, int rmax, bool& bad, uint32_t& ph) {
    const int tid = static_cast<int>(threadIdx.x), lane = tid & 31, warp = tid >> 5;
    const double2 zero = make_double2(0.0, 0.0);
    // scratch behind the 7 B planes of the product: Z (then X) and the pivots' reciprocals
    double2* Zs = reinterpret_cast<double2*>(T.b + kTD * kPlaneS);   // [c][m]
    double2* inv = Zs + kNB * kNB;
    static_assert((kNB * kNB + kNB) * static_cast<int>(sizeof(double2)) <= kTD * kPlaneS,
                  "panel scratch fits behind the B planes");
    // (1) pair p < 120 of the pairs with jp >= 1: jp = 15 (1 pair), 14 (2), ...
    int jp = -1, i = -1;
    if (tid < kNB * (kNB - 1) / 2) {
        int base = 0, c = kNB - 1;
        while (tid >= base + (kNB - c)) {
            base += kNB - c;
            --c;
        }
        jp = c;
        i = c + (tid - base);
    }
    const int sc = tid - 128;   // the scaling threads 128 .. 143: row sc of the column before
    for (int j = 0; j < kNB; ++j) {
        const double2 D = P[j * RP + j];
        if (tid == 0 && (!(fabs(D.x) + fabs(D.y) > 0.0) || !isfinite(D.x) || !isfinite(D.y))) bad = true;
        if (jp > j) {
            const double2 r = j == 0 ? crecip(D) : inv[j];
            const double2 l = cmul(P[j * RP + i], r);
            const double2 t = cfms(P[jp * RP + i], l, P[j * RP + jp]);
            P[jp * RP + i] = t;
            if (i == jp && jp == j + 1) inv[jp] = crecip(t);   // the next pivot is final
        }
        if (j == 0 && sc == 0) inv[0] = crecip(D);
        if (j > 0 && sc > j - 1 && sc < kNB) P[(j - 1) * RP + sc] = cmul(P[(j - 1) * RP + sc], inv[j - 1]);
        __syncthreads();
    }
    // (2) X = L11^{-1}: half warp m (tid >> 4) holds column m, lane c = tid & 15 the entry X[c][m];
    // then Z[m][c] = X[c][m] / D_c and the B scales (a thread per column c)
    if (tid < kNB * kNB) {
        const int m = tid >> 4, c = tid & 15, half = tid & 16;
        double2 x = c == m ? make_double2(1.0, 0.0) : zero;
        for (int k = 2 * (warp); k < kNB - 1; ++k) {   // columns m < 2 warp + 2 start at k = m
            const double2 xk = shfl_c(x, half | k);
            if (c > k && k >= m) x = cfms(x, P[k * RP + c], xk);
        }
        Zs[c * kNB + m] = c >= m ? cmul(x, inv[c]) : zero;
    }
    __syncthreads();
    if (tid < kNB) {
        int e = tc::kNoExp;
        for (int m = 0; m < kNB; ++m) {
            const double2 z = Zs[tid * kNB + m];
            e = max(e, max(tc::exp_of(z.x), tc::exp_of(z.y)));
        }
        T.tb[tid] = scale_of(e);
    }
    __syncthreads();
    // (3) B digits (256 threads, 4 K each: part, column c, K quarter-group kq)
    if (tid < 2 * kSN * 8) {
        const int part = tid >> 7, u = tid & 127;
        const int c = u & 15, kq = u >> 4, kg = kq >> 1;
        const int Tb = T.tb[c];
        unsigned long long U[4];
        bool neg[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double2 z = Zs[c * kNB + ((4 * kq + q) & 15)];
            double x;
            if (part == 0) x = kg < 2 ? z.x : neg_bits(z.y);
            else x = kg < 2 ? z.y : z.x;
            U[q] = tc::to_fixed_mag(x, Tb, neg[q]);
        }
        const int mb = 8 * (c >> 2) + 4 * part + (c & 3);
        put_digits4(U, neg, T.b, kPlaneS, core_off(mb, kg) + (kq & 1) * 8);
    }
    const int rows = rmax - kNB;   // rows kNB .. rmax - 1
    for (int m0 = 0; m0 < rows; m0 += kTM) {
        {   // A: four threads per row (four panel columns each) agree on the row's scale
            const int m = tid >> 2, part = tid & 3;
            const int r = kNB + m0 + m;
            double2 a[4];
            int e = tc::kNoExp;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = m0 + m < rows ? P[(4 * part + q) * RP + r] : zero;
                e = max(e, max(tc::exp_of(a[q].x), tc::exp_of(a[q].y)));
            }
            e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
            e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
            const int Ta = scale_of(e);
            if (part == 0) T.ta[m] = Ta;
            unsigned long long U[4];
            bool neg[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) U[q] = tc::to_fixed_mag(a[q].x, Ta, neg[q]);
            put_digits4(U, neg, T.a, kPlaneA, core_off(m, part >> 1) + (part & 1) * 8);
#pragma unroll
            for (int q = 0; q < 4; ++q) U[q] = tc::to_fixed_mag(a[q].y, Ta, neg[q]);
            put_digits4(U, neg, T.a, kPlaneA, core_off(m, 2 + (part >> 1)) + (part & 1) * 8);
        }
        tc::fence_async_shared();
        tc::tc_fence_before_sync();
        __syncthreads();
        if (tid == 0 && !T.fail) {
            tc::tc_fence_after_sync();
            issue_levels<2 * kSN, kPlaneA, kPlaneS>(T.tmem, tc::smem_desc(tc::smem_addr(T.a), 128, 512),
                                                    tc::smem_desc(tc::smem_addr(T.b), 128, 512));
            tc::mma_commit(&T.bar[0]);
        }
        bool ok = true;
        if (!T.fail) ok = tc::mbar_wait(&T.bar[0], ph & 1u);
        ph ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) T.fail = 1;
            return false;
        }
        tc::tc_fence_after_sync();
        {   // rows m = 32 (warp & 3) + lane, columns c = 4 (warp >> 2) ...: L21 = the rounded sums
            const int ql = warp & 3, g = warp >> 2;
            const int m = 32 * ql + lane;
            const uint32_t trow = T.tmem + (static_cast<uint32_t>(32 * ql) << 16) + 8 * g;
            long long Qr[4], Qi[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) Qr[k] = Qi[k] = 0;
#pragma unroll
            for (int l0 = 2; l0 <= kTNL; l0 += 2) {
                uint32_t v[2][8];
#pragma unroll
                for (int u = 0; u < 2; ++u) tc::tmem_ld8_async(trow + (l0 + u - 2) * (2 * kSN), v[u]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    add_level_pair(Qr[k], level_int(v[0][k]), level_int(v[1][k]), l0);
                    add_level_pair(Qi[k], level_int(v[0][4 + k]), level_int(v[1][4 + k]), l0);
                }
            }
            if (m0 + m < rows) {
                const int r = kNB + m0 + m;
                const int Ta = T.ta[m];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c = 4 * g + k;
                    const int E = Ta + T.tb[c] - 54;
                    P[c * RP + r] = make_double2(tc::fixed_to_double(Qr[k], E), tc::fixed_to_double(Qi[k], E));
                }
            }
        }
        tc::tc_fence_before_sync();
        __syncthreads();   // TMEM and the A planes are reused by the next tile
    }
    return true;
}

// Matrix qi of the launch: assembly and blocked band L D L^T into its band buffer (column k: D_k
// at d = 0, L_{k+d,k} at d >= 1).  Sets bad on a vanishing or non-finite pivot.  TC: the trailing
// updates run on the tensor cores (T: the block's tensor-core state, ph its mbarrier phase).
template <bool TC>
__device__ void factor_matrix(const LatticeArgs& A, int q0, int qi, unsigned char* smem, bool& bad,
                              TcSmem* T, uint32_t& ph) {
    int sp, n;
    item_of(A, q0 + qi, sp, n);
    const int N = A.N, b = A.b, S = b + 1, RP = panel_stride(b);
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
        const int rmax = min(kNB + b, N - k0);       // rows k0 .. k0 + rmax - 1 exist
        // (a) stage the panel, zero outside each column's band
        for (int j = warp; j < kNB; j += kWarps)
            for (int i = lane; i < RP; i += 32) {
                double2 v = zero;
                if (j < nb && i >= j && i - j <= b && i < rmax)
                    v = Bq[static_cast<size_t>(k0 + j) * S + (i - j)];
                P[j * RP + i] = v;
            }
        __syncthreads();
        // (b) factor it: column j -> L (scaled by 1/D_j); A[i][j'] -= L_ij v_j' (v = D_j L_j'j);
        //     full panels with rows below their diagonal block on the tensor cores (TC)
        bool panel_done = false;
        if constexpr (TC) {
            if (nb == kNB && rmax > kNB && !T->fail) panel_done = panel_tc(*T, P, RP, rmax, bad, ph);
        }
        for (int j = 0; j < nb && !panel_done; ++j) {
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
        if constexpr (TC) {
            if (nb == kNB) {   // full panels; the last, narrower one (and small tails) below
                trailing_tc(*T, P, RP, nb, tend, Bq, k0, S, ph);
                __syncthreads();
                continue;
            }
        }
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

// The same forward solves with the bulk of each 16-column step on the tensor cores (128 <= b <=
// kTcMaxBand).  Step J: (i) the panel's own triangle (DFMA, in registers), which finishes
// y_J .. y_{J+15} and adds their y^2 / D to G; (ii) they are cut into the digits of
// B_re = [Re y | -Im y], B_im = [Im y | Re y] (16 right-hand sides, K = 32; a plane holds both,
// interleaved by fours: row 8 (r / 4) + 4 part + r % 4) and their slots freed for the indices
// J + S .. J + S + 15; (iii) the rows J + 16 .. J + 15 + b lose sum_j L_rj y_j, formed as in
// trailing_tc with A = [Re L | Im L] (128 rows per tile) and 32 TMEM columns per level (eight
// levels: 256 columns), and subtracted from their window slots.

__device__ void solve_chunk_tc(const LatticeArgs& A, int q0, int qi, int ch, unsigned char* smem,
                               TcSmem& T, uint32_t& ph) {
    int sp, n;
    item_of(A, q0 + qi, sp, n);
    const int N = A.N, b = A.b, S = b + 1;
    const int tid = static_cast<int>(threadIdx.x), lane = tid & 31, warp = tid >> 5;
    const double2 zero = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
    const double2* Bq = A.scratch + static_cast<size_t>(qi) * N * S;
    const int* pos = A.wide_pos + static_cast<size_t>(sp) * A.wide_npos + ch * kR;
    const int* out = A.wide_out + static_cast<size_t>(sp) * A.wide_npos + ch * kR;
    const int nr = min(kR, A.wide_npos - ch * kR);
    double2* Y = reinterpret_cast<double2*>(smem);   // [kR][S], index j in slot j mod S
    const int j0 = pos[0];
    for (int e = tid; e < kR * S; e += kT) Y[e] = zero;
    __syncthreads();
    if (tid < nr && pos[tid] - j0 < S) Y[tid * S + pos[tid] % S] = one;
    // the panel's L triangle, Lp[16 jj + i] = L_{J+i, J+jj} (i > jj), and 1 / D_{J+jj} at i = jj:
    // the 256 entries behind the windows
    double2* Lp = Y + kR * S;
    // thread (rhs r = tid >> 4, panel row i = tid & 15), tid < 256: the position of its
    // right-hand side, and sum_i y_i^2 / D_i over its panel rows (the 16 partial sums of a
    // right-hand side are added at the end)
    const int pr = (tid < kR * kNB && (tid >> 4) < nr) ? pos[tid >> 4] : -1;
    double2 acc = zero;
    for (int J = j0; J < N; J += kNB) {
        const int nb = min(kNB, N - J);
        const int rows = min(b, N - J - nb);   // rows J + nb .. J + nb + rows - 1 below the panel
        const bool bulk = nb == kNB && rows > 0 && !T.fail;
        if (tid < kNB * kNB) {
            const int jj = tid >> 4, i = tid & 15;
            if (jj < nb && i < nb && i >= jj) {
                const double2 l = __ldcg(Bq + static_cast<size_t>(J + jj) * S + (i - jj));
                Lp[tid] = i == jj ? crecip(l) : l;
            }
        }
        __syncthreads();
        // (i) the panel's triangle in registers, y_{J+jj} of a right-hand side passed along its
        // half warp by shuffle; (ii) its B digits straight from the registers; then the panel's
        // window slots take the indices J + S ...  No barrier: the next one (before the MMAs) also
        // publishes the digits, and each thread touches only its own slot.
        if (tid < kR * kNB) {
            const int r = tid >> 4, i = tid & 15, half = tid & 16;
            const int si = (J + i) % S;
            double2 y = i < nb ? Y[r * S + si] : zero;
            for (int jj = 0; jj < nb; ++jj) {
                const double2 yj = shfl_c(y, half | jj);
                if (i > jj && i < nb) y = cfms(y, Lp[16 * jj + i], yj);
            }
            if (i < nb) {
                acc = cfma(acc, cmul(y, y), Lp[17 * i]);
                Y[r * S + si] = (J + i + S == pr) ? one : zero;
            }
            if (bulk) {
                int e = max(tc::exp_of(y.x), tc::exp_of(y.y));   // the row's scale: its half warp
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
                const int Tb = scale_of(e);
                if (i == 0) T.tb[r] = Tb;   // for the epilogues
                // lane i = 4 a + c cuts K quad a of part c: B_re = [Re y | -Im y] (c = 0, 1),
                // B_im = [Im y | Re y] (c = 2, 3)
                const int a = i >> 2, c = i & 3;
                unsigned long long U[4];
                bool neg[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double2 v = shfl_c(y, half | (4 * a + q));
                    const double x = c == 0 ? v.x : c == 1 ? -v.y : c == 2 ? v.y : v.x;
                    U[q] = tc::to_fixed_mag(x, Tb, neg[q]);
                }
                const int kq = (c & 1) * 4 + a;
                const int mb = 8 * (r >> 2) + 4 * (c >> 1) + (r & 3);
                put_digits4(U, neg, T.b, kPlaneS, core_off(mb, kq >> 1) + (kq & 1) * 8);
            }
        }
        // no rows below a short last panel; after a failed MMA wait the block does no more
        // tensor-core work (the launch reports HF_ETIMEOUT)
        if (!bulk) {
            __syncthreads();   // Lp is restaged by the next panel
            continue;
        }
        // (iii) rows below, 128 per tile.  A: the rows' L entries, four threads per row (four panel
        // columns each, adjacent lanes); the next tile's are loaded while this tile's MMAs run,
        // from clamped positions (the entries outside the band zeroed at use)
        const int am = tid >> 2, apart = tid & 3;
        double2 lnext[4];
        const auto load_rows = [&](int mt) {
            const int r = J + nb + min(mt + am, rows - 1);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jj = 4 * apart + q;
                lnext[q] = __ldcg(Bq + static_cast<size_t>(J + jj) * S + min(r - (J + jj), b));
            }
        };
        load_rows(0);
        for (int m0 = 0; m0 < rows; m0 += kTM) {
            {   // the rows agree on their scales by shuffle and cut the Re and Im digits
                const int m = am, part = apart;
                const int r = J + nb + m0 + m;
                double2 l[4];
                int e = tc::kNoExp;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jj = 4 * part + q, d = r - (J + jj);
                    l[q] = (m0 + m < rows && d <= b) ? lnext[q] : zero;
                    e = max(e, max(tc::exp_of(l[q].x), tc::exp_of(l[q].y)));
                }
                e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
                e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
                const int Ta = scale_of(e);
                if (part == 0) T.ta[m] = Ta;
                unsigned long long U[4];
                bool neg[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) U[q] = tc::to_fixed_mag(l[q].x, Ta, neg[q]);
                put_digits4(U, neg, T.a, kPlaneA, core_off(m, part >> 1) + (part & 1) * 8);
#pragma unroll
                for (int q = 0; q < 4; ++q) U[q] = tc::to_fixed_mag(l[q].y, Ta, neg[q]);
                put_digits4(U, neg, T.a, kPlaneA, core_off(m, 2 + (part >> 1)) + (part & 1) * 8);
            }
            tc::fence_async_shared();
            tc::tc_fence_before_sync();
            __syncthreads();
            if (tid == 0 && !T.fail) {
                tc::tc_fence_after_sync();
                issue_levels<2 * kSN, kPlaneA, kPlaneS>(T.tmem, tc::smem_desc(tc::smem_addr(T.a), 128, 512),
                                                        tc::smem_desc(tc::smem_addr(T.b), 128, 512));
                tc::mma_commit(&T.bar[0]);
            }
            if (m0 + kTM < rows) load_rows(m0 + kTM);
            bool ok = true;
            if (!T.fail) ok = tc::mbar_wait(&T.bar[0], ph & 1u);
            ph ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) T.fail = 1;
                break;
            }
            tc::tc_fence_after_sync();
            {   // lane quarter (warp & 3): rows m = 32 (warp & 3) + lane; warp >> 2: rhs 4 g ...
                // 4 g + 3, their Re and Im sums side by side
                const int ql = warp & 3, g = warp >> 2;
                const int m = 32 * ql + lane;
                const uint32_t trow = T.tmem + (static_cast<uint32_t>(32 * ql) << 16) + 8 * g;
                long long Qr[4], Qi[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) Qr[k] = Qi[k] = 0;
#pragma unroll
                for (int l0 = 2; l0 <= kTNL; l0 += 2) {
                    uint32_t v[2][8];
#pragma unroll
                    for (int u = 0; u < 2; ++u) tc::tmem_ld8_async(trow + (l0 + u - 2) * (2 * kSN), v[u]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        add_level_pair(Qr[k], level_int(v[0][k]), level_int(v[1][k]), l0);
                        add_level_pair(Qi[k], level_int(v[0][4 + k]), level_int(v[1][4 + k]), l0);
                    }
                }
                if (m0 + m < rows) {
                    const int r = J + nb + m0 + m, sr = r % S;
                    const int Ta = T.ta[m];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int rh = 4 * g + k;
                        const int E = Ta + T.tb[rh] - 54;
                        double2* y = Y + rh * S + sr;
                        const double2 x = *y;
                        *y = make_double2(x.x - tc::fixed_to_double(Qr[k], E), x.y - tc::fixed_to_double(Qi[k], E));
                    }
                }
            }
            tc::tc_fence_before_sync();
            __syncthreads();
        }
    }
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (tid < kR * kNB && (tid & 15) == 0 && (tid >> 4) < nr) {
        A.gloc[static_cast<size_t>(out[tid >> 4]) * A.nw + n] = acc;
        if (!isfinite(acc.x) || !isfinite(acc.y)) atomicExch(A.status, static_cast<int>(HF_ENUMERIC));
    }
}

// One persistent block per SM.  The tasks of a launch are the nq factorisations, then the
// nq * nchunk solve tasks (matrix-major); blocks take them in order from work[0].  A block that
// finishes a factorisation raises work[1 + qi]; a solve task waits for its matrix's flag (it was
// handed out earlier, so a running block is factoring it), at most wait_cycles (several times
// what one factorisation takes), after which it reports HF_ETIMEOUT and skips.  So the blocks
// left over when the factorisations run out take the solves of the matrices already factored,
// instead of idling through a last partial wave.  TC: the block holds all of TMEM and the
// mbarriers of the tensor-core products (one per warp group of the trailing update), from its
// first task to its last.
template <int DPT, bool TC>
__global__ void __launch_bounds__(kT, 1) lattice_wide_kernel(const LatticeArgs A, int q0, int nq,
                                                             int nchunk, int* work,
                                                             long long wait_cycles) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int task_s, ready_s;
    const int tid = static_cast<int>(threadIdx.x);
    const int ntask = nq * (1 + nchunk);
    bool bad = false;
    TcSmem* T = nullptr;
    uint32_t ph = 0u;
    if constexpr (TC) {
        T = reinterpret_cast<TcSmem*>(smem + tc_offset_dev(A.b));
        if (tid == 0) {
            T->fail = 0;
            for (int g = 0; g < 4; ++g) tc::mbar_init(&T->bar[g], 1);   // one commit per tile
            tc::mbar_init_fence();
        }
        if (tid < 32) tc::tmem_alloc(&T->tmem, 512);
        tc::tc_fence_before_sync();
        __syncthreads();
        tc::tc_fence_after_sync();
    }
    for (;;) {
        if (tid == 0) task_s = atomicAdd(work, 1);
        __syncthreads();
        const int t = task_s;
        if (t >= ntask) break;
        if (t < nq) {
            factor_matrix<TC>(A, q0, t, smem, bad, T, ph);
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
            if (ready_s) {
                if constexpr (TC) solve_chunk_tc(A, q0, qi, ch, smem, *T, ph);
                else solve_chunk<DPT>(A, q0, qi, ch, smem);
            }
            else if (tid == 0) atomicExch(A.status, static_cast<int>(HF_ETIMEOUT));
        }
        __syncthreads();                             // task_s and the shared memory are reused
    }
    if constexpr (TC) {
        __syncthreads();
        tc::tc_fence_after_sync();
        if (tid < 32) tc::tmem_dealloc(T->tmem, 512);
        if (tid == 0 && T->fail) atomicExch(A.status, static_cast<int>(HF_ETIMEOUT));
    }
    if (bad) atomicExch(A.status, static_cast<int>(HF_ENUMERIC));
}

}  // namespace

int lattice_wide_max_band() { return kWideMaxBand; }

int lattice_wide_tc_min_band() { return kTcMinBand; }

int lattice_wide_rhs_per_block() { return kR; }

double lattice_wide_tc_flops(int N, int b, const int* pos, int npos, int nspin) {
    if (b < kTcMinBand || b > kTcMaxBand) return 0.0;
    // one tile of 128 rows with W columns on the B side: 2 flops x 2 K halves x the digit pairs
    // of levels <= kTNL x 128 x W x 16
    int pairs = 0;
    for (int sd = 1; sd <= kTD; ++sd)
        for (int td = 1; td <= kTD; ++td)
            if (sd + td <= kTNL) ++pairs;
    const double tile32 = 4.0 * pairs * kTM * (2 * kSN) * 16;
    const double tile_rt = 4.0 * pairs * kTM * (2 * kRT) * 16;
    double f = 0.0;
    for (int k0 = 0; k0 + kNB <= N; k0 += kNB) {   // full panels
        const int rmax = std::min(kNB + b, N - k0);
        // the rows below the diagonal block: tiles of 128 with the 16 columns of Z
        f += tile32 * ((rmax - kNB + kTM - 1) / kTM);
        // the trailing update: column tiles of 128, row tiles of kRT from the tile's first column on
        const int rows = std::min(kNB - 1 + b, rmax - 1) - kNB + 1;
        for (int c0 = 0; c0 < rows; c0 += kTM) f += tile_rt * ((rows - c0 + kRT - 1) / kRT);
    }
    // the forward solves: per task of kR positions (ascending), from its first position, the rows
    // below each full step in tiles of 128
    double sv = 0.0;
    for (int sp = 0; sp < nspin; ++sp)
        for (int ch = 0; ch * kR < npos; ++ch) {
            const int j0 = pos[static_cast<size_t>(sp) * npos + ch * kR];
            for (int J = j0; J + kNB <= N; J += kNB) {
                const int rows = std::min(b, N - J - kNB);
                if (rows > 0) sv += tile32 * ((rows + kTM - 1) / kTM);
            }
        }
    return f + sv / std::max(nspin, 1);
}

cudaError_t launch_lattice_wide(const LatticeArgs& a, int q0, int nq, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    if (a.b < 0 || a.b > kWideMaxBand || a.wide_npos <= 0 || !a.wide_pos || !a.wide_out || !a.work)
        return cudaErrorInvalidValue;
    const bool one = a.b <= kT;
    const bool tcu = a.b >= kTcMinBand && a.b <= kTcMaxBand;
    auto kern = tcu ? (one ? lattice_wide_kernel<1, true> : lattice_wide_kernel<2, true>)
                    : (one ? lattice_wide_kernel<1, false> : lattice_wide_kernel<2, false>);
    const size_t smax = std::max(wide_smem(kWideMaxBand, false), wide_smem(kTcMaxBand, true));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smax));
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
    kern<<<grid, kT, wide_smem(a.b, tcu), st>>>(a, q0, nq, nchunk, a.work, wait);
    return cudaGetLastError();
}

}  // namespace hfk
