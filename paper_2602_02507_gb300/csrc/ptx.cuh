// ptx.cuh -- inline-PTX wrappers for sm_103a: mbarrier, TMA (cp.async.bulk),
// tcgen05 (tensor memory, UMMA issue, commit, loads) and bit-level float
// conversions that avoid the float64 pipe.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>

#include "mp_errors.h"

namespace mp {

// A wait on an mbarrier gives up after this many SM clock cycles (about a
// second at the GB300 boost clock) and reports DEV_ERR_TIMEOUT.
#ifndef MP_WAIT_BUDGET_CYCLES
#define MP_WAIT_BUDGET_CYCLES (2000000000LL)
#endif

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait.  Returns false (after raising the CTA's abort flag and the
// mesh error word) when the phase does not complete within the budget, or
// when another role of the CTA already aborted.
// The mesh's device error word is err[0]; err[2..3] hold, as one 64-bit value, the
// budget of these pipeline waits in SM clock cycles (0 or less: MP_WAIT_BUDGET_CYCLES;
// mp_set_wait_budget changes it).  The drains that follow an abort always keep the
// full compile-time budget, so that no copy or MMA outlives the block that issued it.
// The budget is written only between launches (the host sets it with the stream idle),
// so it is read through the read-only data cache: a volatile read of it in every wait
// that does not complete at once cost the projection and the phi synthesis about 20 us
// each per solve of 2048 x 512 x 1024 cells.
__device__ __forceinline__ long long wait_budget(const int *err)
{
    const long long b = __ldg(reinterpret_cast<const long long *>(err + 2));
    return b > 0 ? b : MP_WAIT_BUDGET_CYCLES;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    const long long budget = wait_budget(err);
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) {
            *abort_flag = 1;
            atomicOr(err, DEV_ERR_TIMEOUT);
            return false;
        }
    }
}

// Position in a ring of mbarrier-guarded stages: index and phase advance together.
struct Ring {
    int idx = 0;
    uint32_t phase = 0;
    __device__ __forceinline__ void next(int n)
    {
        if (++idx == n) {
            idx = 0;
            phase ^= 1u;
        }
    }
    __device__ __forceinline__ void prev(int n)
    {
        if (idx == 0) {
            idx = n;
            phase ^= 1u;
        }
        --idx;
    }
};

// After an abort: waits (bounded by the full budget) for the last min(n, issued) copies
// issued into the n-slot ring whose next free position is r, so that none of them is still
// writing into this block's shared memory when the block exits.
__device__ __forceinline__ void drain_ring(uint64_t *full, Ring r, int n, int issued)
{
    for (int k = 0; k < n && k < issued; ++k) {
        r.prev(n);
        const long long t0 = clock64();
        while (!mbar_try_wait(smem_u32(&full[r.idx]), r.phase) && clock64() - t0 < MP_WAIT_BUDGET_CYCLES) {
        }
    }
}

// Tensor-memory allocation size: a power of two of at least 32 columns.
__device__ __forceinline__ uint32_t tmem_ncols_for(int cols)
{
    uint32_t n = 32;
    while (n < (uint32_t)cols) n <<= 1;
    return n;
}

__device__ __forceinline__ bool warp_all(bool v) { return __all_sync(0xFFFFFFFFu, v); }

// ---------------------------------------------------------------- programmatic dependent launch
// Blocks until the grids this one depends on (the previous kernel on the
// stream, when launched with programmatic stream serialization) have completed
// and their memory is visible; returns at once otherwise.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Lets the next kernel on the stream start its blocks once every block of this
// grid has issued the trigger or exited (so a block of this grid never waits
// for resources held by waiting dependents); they still wait in pdl_wait for
// this grid to complete.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// ---------------------------------------------------------------- TMA / bulk copies
__device__ __forceinline__ void tma_prefetch_desc(const void *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void *map, uint32_t bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const void *map, uint32_t src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}

// L2 policy for data touched once (a stream read or written once per solve): its lines are
// the first to be evicted, so they neither displace reused data nor linger dirty in L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const void *map, uint32_t bar, int x, int y,
                                                 uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void tma_store_2d_hint(const void *map, uint32_t src, int x, int y, uint64_t policy)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group.L2::cache_hint [%0, {%2, %3}], [%1], %4;"
                 ::"l"(map), "r"(src), "r"(x), "r"(y), "l"(policy)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_read_le1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_read_le3() { asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Per-thread asynchronous copies global -> shared (cp.async, not the bulk engine): src_bytes
// below the copy size fill the rest with zeros (0: nothing is read).  A thread sees its own
// copies after cp_async_wait<N> leaves at most N of its committed groups pending; other
// threads' copies need a barrier after that wait as well.
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async4_zfill(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, fp32 accumulate, one thread issues.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on the mbarrier when every tcgen05 op issued so far by this thread is done.
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 32 lanes x 8 / 16 consecutive 32-bit columns; thread t of the warp gets lane
// (32 * (warp % 4) + t) of the addressed lane quarter.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// 8-row x 16-byte core matrices; lbo = byte step between the two core matrices
// adjacent along K, sbo = byte step between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t sdesc_noswizzle(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16;
    d |= static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32;
    d |= static_cast<uint64_t>(1) << 46;  // descriptor version field of tcgen05
    return d;                             // base offset 0, relative LBO, layout type 0 (no swizzle)
}

// Instruction descriptor of tcgen05.mma kind::f16: bf16 x bf16 -> fp32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4)                                 // D format fp32
           | (1u << 7)                               // A format bf16
           | (1u << 10)                              // B format bf16
           | (static_cast<uint32_t>(N >> 3) << 17)   // N / 8
           | (static_cast<uint32_t>(M >> 4) << 24);  // M / 16
}

// ---------------------------------------------------------------- bit conversions
// float64 (as two 32-bit words) -> float32, round-half-up on the 29 dropped
// mantissa bits, integer ops only.  Magnitudes below the float32 normal range
// flush to zero, above it saturate to infinity.
__device__ __forceinline__ float f64w_to_f32(uint32_t lo, uint32_t hi)
{
    const uint32_t sign = hi & 0x80000000u;
    const int e = static_cast<int>((hi >> 20) & 0x7FFu) - 896;
    const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    uint32_t bits = (static_cast<uint32_t>(e) << 23) + mant + ((lo >> 28) & 1u);
    bits = (e <= 0) ? 0u : bits;
    bits = (e >= 255) ? 0x7F800000u : bits;
    return __uint_as_float(bits | sign);
}

__device__ __forceinline__ bool f64w_nonfinite(uint32_t hi) { return (hi & 0x7FF00000u) == 0x7FF00000u; }

// Same conversion, cheaper, for values that are split into bf16 terms next
// (which keep about 16 significant bits): the float32 exponent field is the low
// eight float64 exponent bits with the top bit flipped (for exponents inside the
// float32 normal range), and the 23 mantissa bits are the top float64 mantissa
// bits with the lowest one forced to 1 ("jamming": at most one float32 ulp from
// the value and, unlike truncation, without a bias toward zero).  Magnitudes
// below 2^-126 (zeros included) give a signed zero.  Magnitudes at or above
// 2^128 (and inf, nan) give no meaningful result: the caller tracks
// ef = hi & 0x7FF00000 (returned) and reports them.
__device__ __forceinline__ float f64w_to_f32_fast(uint32_t lo, uint32_t hi, uint32_t &ef)
{
    const uint32_t t = __funnelshift_l(lo, hi, 3);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t r = (((t & 0x7FFFFFFFu) | sign) ^ 0x40000000u) | 1u;
    ef = hi & 0x7FF00000u;
    return __uint_as_float(ef >= (897u << 20) ? r : sign);
}

// The same conversion for a magnitude known to lie in float32's normal range (no
// range select): the caller checks the range on its own.
__device__ __forceinline__ float f64w_to_f32_inrange(uint32_t lo, uint32_t hi)
{
    const uint32_t t = __funnelshift_l(lo, hi, 3);
    return __uint_as_float((((t & 0x7FFFFFFFu) | (hi & 0x80000000u)) ^ 0x40000000u) | 1u);
}

// float64 -> float32 with integer ops (round to nearest, ties away from zero):
// magnitudes below float32's normal range give signed zero, above it signed
// infinity (so do inf and nan).
__device__ __forceinline__ float f64_to_f32_alu(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t hi = static_cast<uint32_t>(b >> 32);
    const uint32_t ef = hi & 0x7FF00000u, sign = hi & 0x80000000u;
    const uint32_t t = static_cast<uint32_t>((b + (1ull << 28)) >> 29);
    uint32_t r = ((t & 0x7FFFFFFFu) | sign) ^ 0x40000000u;
    r = (ef < (897u << 20)) ? sign : r;
    r = (ef > (1150u << 20)) ? (sign | 0x7F800000u) : r;
    return __uint_as_float(r);
}

// float32 -> float64 words, exact for normal numbers, integer ops only.
__device__ __forceinline__ void f32_to_f64w(float x, uint32_t &lo, uint32_t &hi)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t mag = b & 0x7FFFFFFFu;
    const uint32_t sign = b & 0x80000000u;
    uint32_t h = ((mag >> 3) + 0x38000000u) | sign;
    uint32_t l = b << 29;
    h = (mag < 0x00800000u) ? sign : h;
    l = (mag < 0x00800000u) ? 0u : l;
    h = (mag >= 0x7F800000u) ? (sign | 0x7FF00000u | ((mag & 0x7FFFFFu) ? 0x80000u : 0u)) : h;
    lo = l;
    hi = h;
}

// float32 -> float64 words for finite x: exact for normal numbers, zero (with
// sign) for zeros and float32 subnormals.  Non-finite inputs are not preserved.
__device__ __forceinline__ void f32_to_f64w_finite(float x, uint32_t &lo, uint32_t &hi)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t sign = b & 0x80000000u;
    const uint32_t mag = b & 0x7FFFFFFFu;
    const uint32_t h = ((mag >> 3) + 0x38000000u) | sign;
    const bool normal = mag >= 0x00800000u;
    hi = normal ? h : sign;
    lo = normal ? (b << 29) : 0u;
}

// float32 -> float64, exact for finite normal inputs (subnormals give zero),
// integer ops only (the float64 pipe stays free).
__device__ __forceinline__ double f32_to_f64_alu(float x)
{
    uint32_t lo, hi;
    f32_to_f64w_finite(x, lo, hi);
    return __hiloint2double((int)hi, (int)lo);
}

// float64 -> (hi, lo) float pair with hi + lo = x to about 2^-48 relative.
__device__ __forceinline__ float2 f32_pair(double x)
{
    const float hi = f64_to_f32_alu(x);
    return make_float2(hi, f64_to_f32_alu(x - f32_to_f64_alu(hi)));
}

// Two float32 subtractions in one packed instruction (each rounded to nearest, as the
// scalar form): a - b for both halves.
__device__ __forceinline__ float2 sub_f32x2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rr;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rr, ra, rb;\n\tmov.b64 {%0, %1}, rr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// Round-to-nearest bf16 pair packed in one word (x in the low half).
__device__ __forceinline__ uint32_t pack_bf16x2(float x, float y)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float bf16lo_to_f32(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi_to_f32(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// The m = 0 column is the bulk of Phi and its Legendre sum can cancel: it is formed in
// double-float arithmetic on the float32 pipe from (hi, lo) pairs of the table T[l] and
// the coefficients c[l] -- products split exactly by fmaf, the running sum kept as a
// TwoSum pair -- and leaves as a (hi, lo) pair (relative error near 2^-44).
__device__ __forceinline__ float2 g0_double_float(const float2 *T, int t_stride, const float2 *c, int L)
{
    float s = 0.0f, e = 0.0f;
    for (int l = 0; l <= L; ++l) {
        const float2 t = T[(size_t)l * t_stride], k = c[l];
        const float p = __fmul_rn(t.x, k.x);
        const float pe = fmaf(t.x, k.x, -p);            // exact error of the leading product
        const float cross = fmaf(t.x, k.y, __fmul_rn(t.y, k.x));
        const float s2 = __fadd_rn(s, p);                 // TwoSum of the running sum and p
        const float bv = __fsub_rn(s2, s);
        const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bv)), __fsub_rn(p, bv));
        s = s2;
        e = __fadd_rn(e, __fadd_rn(se, __fadd_rn(pe, cross)));
    }
    const float hi = __fadd_rn(s, e);
    return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

// The same sum for NS coefficient rows c + k c_stride (k < NS) sharing the table column T:
// NS independent accumulation chains in flight (a single chain is bound by the latency of
// its dependent float32 operations).
template <int NS>
__device__ __forceinline__ void g0_double_float_n(const float2 *T, int t_stride, const float2 *c, int c_stride, int L,
                                                  float2 (&out)[NS])
{
    float s[NS], e[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) s[k] = e[k] = 0.0f;
    for (int l = 0; l <= L; ++l) {
        const float2 t = T[(size_t)l * t_stride];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            const float2 kk = c[(size_t)k * c_stride + l];
            const float p = __fmul_rn(t.x, kk.x);
            const float pe = fmaf(t.x, kk.x, -p);
            const float cross = fmaf(t.x, kk.y, __fmul_rn(t.y, kk.x));
            const float s2 = __fadd_rn(s[k], p);
            const float bv = __fsub_rn(s2, s[k]);
            const float se = __fadd_rn(__fsub_rn(s[k], __fsub_rn(s2, bv)), __fsub_rn(p, bv));
            s[k] = s2;
            e[k] = __fadd_rn(e[k], __fadd_rn(se, __fadd_rn(pe, cross)));
        }
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const float hi = __fadd_rn(s[k], e[k]);
        out[k] = make_float2(hi, __fsub_rn(e[k], __fsub_rn(hi, s[k])));
    }
}

}  // namespace mp
