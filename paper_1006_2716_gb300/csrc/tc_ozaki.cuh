// tc_ozaki.cuh -- FP64-accurate products of 128 x 128 matrices on the sm_103a tensor cores.
//
// A product C = A B of FP64 matrices is formed from exact integer products (Ozaki, Ogita, Oishi
// and Rump's error-free splitting of a matrix product): every row of A (every column of B) gets
// a power-of-two scale 2^T with |x| <= 2^(T-1), its entries become 62-bit fixed-point integers,
// and those are cut into balanced base-256 digits d_1, d_2, ... in [-128, 128], so that
// x = 2^T sum_s d_s 2^(-8 s) up to the last digit.  A digit is exact in bf16, a product of two
// digits is at most 2^14 and a sum of 128 of them at most 2^21; the sum over the pairs (s, t) of
// one level n = s + t (at most 8 pairs for n <= 9) therefore stays within 2^24, where FP32 is
// exact.
// So each level D_n = sum_{s+t=n} A_s B_t is one tensor-core accumulator in TMEM (tcgen05.mma,
// kind::f16, bf16 operands from shared memory, FP32 accumulation), read back with tcgen05.ld and
// combined in 64-bit integers: C = 2^(Ta_i + Tb_j) sum_n D_n 2^(-8 n).  Levels above the last one
// kept are dropped; with d digits and levels up to d + 1 the product is accurate to about
// 2^(9 - 8 d) of 2^(Ta_i + Tb_j).
//
// This header holds the PTX of the tensor-memory allocator, the MMA, its commit to an mbarrier,
// the TMEM loads and the fences between the thread and async proxies, the shared-memory matrix
// descriptors (K-major, no swizzle: 8-row x 16-byte core matrices) and the integer helpers that
// move between FP64, fixed point and digits without touching the FP64 pipe.
#pragma once

#include <stdint.h>

namespace hfk {
namespace tc {

// ------------------------------------------------------------------------------------------
// shared-memory addresses, mbarriers, proxy fences
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the barrier initialisation visible to the async proxy (the tensor cores arrive on it).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One bounded probe of the barrier's phase with parity `phase`; true once it has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Waits for the phase for at most about 2^31 SM clock cycles (about a second; the tensor-core
// work a wait covers takes microseconds); false if that bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}

// One arrival on the barrier that also announces `bytes` of asynchronous copies still to land
// on it (the phase completes when both have happened).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy (the TMA engine, no tensor map) of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to shared memory, completing on the barrier's transaction count.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Generic-proxy writes to shared memory made visible to the async proxy (the MMA operands).
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------------------------------
// tensor memory
// ------------------------------------------------------------------------------------------
// Allocates ncols (a power of two, 32..512) TMEM columns for the CTA; one whole warp executes it
// and the base address is written to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] B[smem]: M x N x 16 bf16 -> FP32, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// The barrier's phase completes once every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ...).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

// 8 consecutive 32-bit columns of this thread's TMEM lane, without waiting: the registers are
// valid after the next tmem_wait_ld().
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
}

// 16 consecutive 32-bit columns of this thread's TMEM lane, without waiting.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// 4 consecutive 32-bit columns of this thread's TMEM lane, without waiting.
__device__ __forceinline__ void tmem_ld4_async(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major) and an FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4)                                  // D: F32
           | (1u << 7)                                // A: BF16
           | (1u << 10)                               // B: BF16
           | (static_cast<uint32_t>(N >> 3) << 17)    // N / 8
           | (static_cast<uint32_t>(M >> 4) << 24);   // M / 16
}

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16 bytes
// stored as 128 contiguous bytes; lbo = bytes between core matrices adjacent along K, sbo =
// bytes between core matrices adjacent along M (or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) |
           (static_cast<uint64_t>(lbo >> 4) << 16) |
           (static_cast<uint64_t>(sbo >> 4) << 32) |
           (1ull << 46);   // descriptor version of this architecture; no swizzle, base offset 0
}

// ------------------------------------------------------------------------------------------
// FP64 <-> fixed point <-> digits on the integer pipe
// ------------------------------------------------------------------------------------------
constexpr int kNoExp = -4096;   // exponent of zero

// floor(log2 |x|) of a normal double (kNoExp for zero; subnormals count as zero).
__device__ __forceinline__ int exp_of(double x) {
    const int e = (__double2hiint(x) >> 20) & 0x7FF;
    return e == 0 ? kNoExp : e - 1023;
}

// round(x e 2^(62 - T)) for a double x and a constant e = me 2^(Ee - 52) (me its 53-bit
// significand), exact product of the significands on the integer pipe; |x e| <= 2^(T-1).
__device__ __forceinline__ long long to_fixed_scaled(double x, unsigned long long me, int Ee, int T) {
    const long long b = __double_as_longlong(x);
    const int e = static_cast<int>((b >> 52) & 0x7FF);
    if (e == 0) return 0;
    const unsigned long long m = (static_cast<unsigned long long>(b) & 0xFFFFFFFFFFFFFull) |
                                 0x10000000000000ull;
    // (m 2^11)(me 2^11) = m me 2^22: its upper 64 bits are m me 2^-42, in [2^62, 2^64)
    const unsigned long long hi = __umul64hi(m << 11, me << 11);
    // x e = m me 2^(e - 1075 + Ee - 52) = hi 2^(42 + e - 1127 + Ee)
    const int sh = (42 + e - 1127 + Ee) + 62 - T;
    unsigned long long v;
    if (sh >= 0) {
        v = hi << sh;
    } else if (sh > -64) {
        v = (hi >> (-sh)) + ((hi >> (-sh - 1)) & 1ull);
    } else {
        v = 0;
    }
    return b < 0 ? -static_cast<long long>(v) : static_cast<long long>(v);
}

// |round(x 2^(62 - T))| and the sign of x, for |x| <= 2^(T-1) (magnitude <= 2^61).
__device__ __forceinline__ unsigned long long to_fixed_mag(double x, int T, bool& neg) {
    const long long b = __double_as_longlong(x);
    neg = b < 0;
    const int e = static_cast<int>((b >> 52) & 0x7FF);
    if (e == 0) return 0ull;
    const unsigned long long m = (static_cast<unsigned long long>(b) & 0xFFFFFFFFFFFFFull) |
                                 0x10000000000000ull;
    const int sh = (e - 1075) + 62 - T;
    if (sh >= 0) return m << sh;
    if (sh > -64) return (m + (1ull << (-sh - 1))) >> (-sh);
    return 0ull;
}

// |round(x e 2^(62 - T))| and the sign of x, e = me 2^(Ee - 52) > 0 (see to_fixed_scaled).
__device__ __forceinline__ unsigned long long to_fixed_scaled_mag(double x, unsigned long long me,
                                                                  int Ee, int T, bool& neg) {
    const long long b = __double_as_longlong(x);
    neg = b < 0;
    const int e = static_cast<int>((b >> 52) & 0x7FF);
    if (e == 0) return 0ull;
    const unsigned long long m = (static_cast<unsigned long long>(b) & 0xFFFFFFFFFFFFFull) |
                                 0x10000000000000ull;
    const unsigned long long hi = __umul64hi(m << 11, me << 11);
    const int sh = (42 + e - 1127 + Ee) + 62 - T;
    if (sh >= 0) return hi << sh;
    if (sh > -64) return (hi >> (-sh)) + ((hi >> (-sh - 1)) & 1ull);
    return 0ull;
}

// The first SD balanced base-256 digits of a fixed-point magnitude u <= 2^61 (value u 2^-62 =
// sum_s d_s 2^(-8 s) + what the dropped digits held, at most half a unit of the last digit):
// 8-bit fields from the top (the eighth is the remaining 6 bits, scaled to weight 2^-64), made
// balanced from the bottom up by borrowing 256 from a field above 128.  d_s in [-127, 128].
template <int SD>
__device__ __forceinline__ void digits_of(unsigned long long u, int (&d)[SD]) {
    if constexpr (SD < 8) u += 1ull << (61 - 8 * SD);   // rounds the truncation to the nearest
    int f[SD];
#pragma unroll
    for (int s = 1; s <= SD; ++s)
        f[s - 1] = s < 8 ? static_cast<int>((u >> (62 - 8 * s)) & 255ull)
                         : static_cast<int>((u & 63ull) << 2);
    int c = 0;
#pragma unroll
    for (int s = SD; s >= 1; --s) {
        const int v = f[s - 1] + c;
        c = v > 128 ? 1 : 0;
        d[s - 1] = c ? v - 256 : v;
    }
}

// FP32 bit pattern of an integer |d| <= 2^22 (exact), through the binade [2^23, 2^24).
__device__ __forceinline__ uint32_t f32bits_of_int(int d) {
    return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f);
}

// Two digits as a bf16x2 word (the upper halves of their FP32 patterns, d0 low), each negated
// where its element is negative (bf16 sign bits).
__device__ __forceinline__ uint32_t bf16x2_digits(int d0, int d1, bool neg0, bool neg1) {
    const uint32_t w = __byte_perm(f32bits_of_int(d0), f32bits_of_int(d1), 0x7632);
    return w ^ ((neg0 ? 0x8000u : 0u) | (neg1 ? 0x80000000u : 0u));
}

// q 2^E as a double (round to nearest on the integer pipe; q = 0 gives 0).
__device__ __forceinline__ double fixed_to_double(long long q, int E) {
    if (q == 0) return 0.0;
    const unsigned long long sign = q < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long a = q < 0 ? static_cast<unsigned long long>(-q) : static_cast<unsigned long long>(q);
    const int lz = __clzll(static_cast<long long>(a));
    const int top = 63 - lz;                                     // a in [2^top, 2^(top+1))
    // 53 significant bits: shift so that the leading one sits at bit 52
    unsigned long long m;
    if (top > 52) {
        const int sh = top - 52;
        m = (a >> sh) + ((a >> (sh - 1)) & 1ull);
    } else {
        m = a << (52 - top);
    }
    int ex = top + E;                                            // value = (m / 2^52) 2^ex
    if (m >> 53) {                                               // rounding carried out
        m >>= 1;
        ++ex;
    }
    if (ex < -1022) return 0.0;                                  // far below any scale in use
    return __longlong_as_double(static_cast<long long>(
        sign | (static_cast<unsigned long long>(ex + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

}  // namespace tc
}  // namespace hfk
