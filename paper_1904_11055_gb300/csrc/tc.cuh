// Blackwell (sm_100 family) primitives in inline PTX: tensor memory (TMEM),
// tcgen05.mma with the A operand in TMEM, mbarriers and TMA bulk tensor loads.
// Every wait is bounded by a clock budget; on expiry it raises a shared abort
// flag so that all warps leave their loops, and the kernel records a timeout.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace ps {
namespace tc {

constexpr long long kWaitBudgetCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int kErrTimeout = 1;

PS_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- TMEM -------------------------------------------------------------------
PS_DEV void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {  // one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
PS_DEV void tmem_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
PS_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // one full warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
PS_DEV void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
PS_DEV void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 8 columns of 32 bits: this thread's lane, columns taddr.col .. +7
PS_DEV void tmem_st8(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
// 32 lanes x 4 columns of 32 bits: this thread's lane, columns taddr.col .. +3
PS_DEV void tmem_st4(uint32_t taddr, const uint32_t* v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
// 32 lanes x 16 columns of 32 bits: this thread's lane, columns taddr.col .. +15
PS_DEV void tmem_st16(uint32_t taddr, const uint32_t* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
PS_DEV void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 columns of 32 bits: this thread's lane, columns taddr.col .. +15
PS_DEV void tmem_ld16(uint32_t taddr, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
PS_DEV void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Elects one lane of a converged warp.  A tcgen05.commit tracks only the MMAs of
// the thread that executes it, so callers elect once and keep the result.
PS_DEV bool elect_one() {
    uint32_t p;
    asm volatile("{\n\t.reg .pred P;\n\telect.sync _|P, 0xffffffff;\n\tselp.u32 %0, 1, 0, P;\n\t}\n" : "=r"(p));
    return p != 0;
}

// ---- descriptors ------------------------------------------------------------
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                        // D format: F32
           | (1u << 7)                      // A format: BF16
           | (1u << 10)                     // B format: BF16
           | ((uint32_t)(N >> 3) << 17)     // N >> 3
           | ((uint32_t)(M >> 4) << 24);    // M >> 4
}

// Shared-memory matrix descriptor, no swizzle, K-major "interleaved" layout of
// 8-row x 16-byte core matrices: lbo = byte step between core matrices that are
// adjacent along K, sbo = byte step between 8-row groups along M/N.
PS_DEV uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for the sm_100 family
    return d;                // base offset 0, swizzle none
}

// D[tmem] (+)= A[tmem] x B[smem]^T  (M = 128 lanes, K = 16)
PS_DEV void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on `bar` once every tcgen05 operation this thread issued so far has completed
PS_DEV void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// ---- mbarriers --------------------------------------------------------------
PS_DEV void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
PS_DEV void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
PS_DEV void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(smem_u32(bar))
                 : "memory");
}
PS_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// try_wait with a suspend-time hint: the thread may sleep (up to the hint, in ns) until the phase completes
PS_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, "
        "p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}
// Non-blocking test of phase `parity` (acquire when it returns true).
PS_DEV bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, "
        "p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar`, giving up after the clock budget or when
// another thread has raised *abort.  Returns false on give-up.
PS_DEV bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > kWaitBudgetCycles) {
            *abort = 1;
            return false;
        }
    }
}

// The same wait taken by every lane of a warp, with a warp-uniform result (so
// that no .sync.aligned instruction is ever reached by part of a warp).
PS_DEV bool mbar_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort) {
    const bool ok = mbar_wait(bar, parity, abort);
    return __all_sync(0xffffffffu, ok);
}

// ---- TMA ----------------------------------------------------------------------
PS_DEV void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
PS_DEV void tma_load_2d(void* dst_smem, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst_smem)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// Untiled bulk copy global -> shared, completing `bytes` of transaction count on `bar` (both addresses
// 16-byte aligned, bytes a multiple of 16).
PS_DEV void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst_smem)),
                 "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
PS_DEV void prefetch_tensormap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

// ---- split of an FP32 value into bf16 hi + lo ---------------------------------
// hi = RN_bf16(v), lo = RN_bf16(v - hi); packs cells (2c, 2c+1) as (low, high) halves.
PS_DEV void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    float ra = a - __low2float(h), rb = b - __high2float(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(ra, rb);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}
// the same for products x*y, with the residual taken from the exact product (one rounding)
PS_DEV void split2_prod(float x0, float y0, float x1, float y1, uint32_t& hi, uint32_t& lo) {
    const float p0 = x0 * y0, p1 = x1 * y1;
    __nv_bfloat162 h = __floats2bfloat162_rn(p0, p1);
    float r0 = fmaf(x0, y0, -__low2float(h)), r1 = fmaf(x1, y1, -__high2float(h));
    __nv_bfloat162 l = __floats2bfloat162_rn(r0, r1);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// The same for two products at once with packed FP32 pairs (sm_100 family):
// (x0 y0, x1 y1) -> hi = RN_bf16 pair, lo = RN_bf16 pair of the exact residuals.
PS_DEV void split2_prod_x2(float x0, float y0, float x1, float y1, uint32_t& hi, uint32_t& lo) {
    asm("{\n\t"
        ".reg .b64 xa, ya, pa, na, ra;\n\t"
        ".reg .f32 p0, p1, r0, r1;\n\t"
        ".reg .b32 h, n0, n1;\n\t"
        "mov.b64 xa, {%2, %3};\n\t"
        "mov.b64 ya, {%4, %5};\n\t"
        "mul.rn.f32x2 pa, xa, ya;\n\t"
        "mov.b64 {p0, p1}, pa;\n\t"
        "cvt.rn.bf16x2.f32 h, p1, p0;\n\t"
        "xor.b32 n1, h, 0x80008000;\n\t"
        "shl.b32 n0, n1, 16;\n\t"
        "and.b32 n1, n1, 0xffff0000;\n\t"
        "mov.b64 na, {n0, n1};\n\t"
        "fma.rn.f32x2 ra, xa, ya, na;\n\t"
        "mov.b64 {r0, r1}, ra;\n\t"
        "cvt.rn.bf16x2.f32 %1, r1, r0;\n\t"
        "mov.b32 %0, h;\n\t"
        "}"
        : "=r"(hi), "=r"(lo)
        : "f"(x0), "f"(x1), "f"(y0), "f"(y1));
}

// hi = RN_bf16 pair of (a, b); lo = RN_bf16 pair of the residuals (a, b) - hi, taken
// with one packed FP32 subtraction (exact: hi is within a factor 2 of each value).
PS_DEV void split2_fast(float a, float b, uint32_t& hi, uint32_t& lo) {
    asm("{\n\t"
        ".reg .b64 xa, ha, ra;\n\t"
        ".reg .b32 h, h0, h1;\n\t"
        ".reg .f32 r0, r1;\n\t"
        "cvt.rn.bf16x2.f32 h, %3, %2;\n\t"
        "shl.b32 h0, h, 16;\n\t"
        "and.b32 h1, h, 0xffff0000;\n\t"
        "mov.b64 xa, {%2, %3};\n\t"
        "mov.b64 ha, {h0, h1};\n\t"
        "sub.rn.f32x2 ra, xa, ha;\n\t"
        "mov.b64 {r0, r1}, ra;\n\t"
        "cvt.rn.bf16x2.f32 %1, r1, r0;\n\t"
        "mov.b32 %0, h;\n\t"
        "}"
        : "=r"(hi), "=r"(lo)
        : "f"(a), "f"(b));
}

// The same for the products (x0 y0, x1 y1), rounded to FP32 first: hi = RN_bf16 pair of
// the products, lo = RN_bf16 pair of (product - hi).  Against the residual of the exact
// product this drops the product's own FP32 rounding (2^-24 relative), far below the
// bf16 rounding of lo (2^-17 of the product).
PS_DEV void split2_prod_fast(float x0, float y0, float x1, float y1, uint32_t& hi, uint32_t& lo) {
    asm("{\n\t"
        ".reg .b64 xa, ya, pa, ha, ra;\n\t"
        ".reg .f32 p0, p1, r0, r1;\n\t"
        ".reg .b32 h, h0, h1;\n\t"
        "mov.b64 xa, {%2, %3};\n\t"
        "mov.b64 ya, {%4, %5};\n\t"
        "mul.rn.f32x2 pa, xa, ya;\n\t"
        "mov.b64 {p0, p1}, pa;\n\t"
        "cvt.rn.bf16x2.f32 h, p1, p0;\n\t"
        "shl.b32 h0, h, 16;\n\t"
        "and.b32 h1, h, 0xffff0000;\n\t"
        "mov.b64 ha, {h0, h1};\n\t"
        "sub.rn.f32x2 ra, pa, ha;\n\t"
        "mov.b64 {r0, r1}, ra;\n\t"
        "cvt.rn.bf16x2.f32 %1, r1, r0;\n\t"
        "mov.b32 %0, h;\n\t"
        "}"
        : "=r"(hi), "=r"(lo)
        : "f"(x0), "f"(x1), "f"(y0), "f"(y1));
}

}  // namespace tc
}  // namespace ps
