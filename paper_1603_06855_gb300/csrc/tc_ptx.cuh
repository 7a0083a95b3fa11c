// Inline-PTX building blocks shared by the tcgen05 kernels (sm_103a): mbarriers with
// bounded waits, TMA tile loads, shared-memory matrix descriptors (K-major, 128-byte
// swizzle), BF16 MMAs into tensor memory, commits, fences and tensor-memory loads, and
// the three-slice bf16 split of an FP32 value.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include "kernels.h"

namespace tcx {

// Polls of mbarrier.try_wait before a wait gives up (a count, not a time: each poll may itself
// suspend the thread for a short, hardware-defined interval).  Far above any legitimate wait.
constexpr long long WAIT_LIMIT = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false (and PC_ETIMEOUT recorded) when the limit expires.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status, long long limit = WAIT_LIMIT) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicCAS(status, 0, PC_ETIMEOUT);
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory byte offset of K-major element k (bf16) of row r inside a tile of 128-byte
// rows laid out with the 128-byte swizzle (tile base 1024-byte aligned): 16-byte chunk
// index XOR (r mod 8).
__device__ __forceinline__ uint32_t sw128_offset(int r, int kbyte) {
  return (uint32_t)(r * 128 + ((((kbyte >> 4) ^ (r & 7)) & 7) << 4) + (kbyte & 15));
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Instruction descriptor: kind::f16, BF16 x BF16 -> FP32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void split3_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  float r = x - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r);
  lo = __float2bfloat16_rn(r - __bfloat162float(mid));
}

// Three bf16 slices of four FP32 values, packed in memory order (two per 32-bit word).
__device__ __forceinline__ void split4_bf16(float a, float b, float c, float d, uint2& hi, uint2& mid, uint2& lo) {
  __nv_bfloat16 h[4], m[4], l[4];
  split3_bf16(a, h[0], m[0], l[0]);
  split3_bf16(b, h[1], m[1], l[1]);
  split3_bf16(c, h[2], m[2], l[2]);
  split3_bf16(d, h[3], m[3], l[3]);
  auto pk = [](__nv_bfloat16 x, __nv_bfloat16 y) {
    return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
  };
  hi = make_uint2(pk(h[0], h[1]), pk(h[2], h[3]));
  mid = make_uint2(pk(m[0], m[1]), pk(m[2], m[3]));
  lo = make_uint2(pk(l[0], l[1]), pk(l[2], l[3]));
}

// Exact three-way split: hi is x rounded to 8 significand bits (to nearest, ties to even, on
// the bit pattern), mid the remainder x - hi rounded the same way, and lo = x - hi - mid,
// which has at most 8 significant bits and so is a bf16 value as it stands: x = hi + mid + lo
// exactly for normal FP32 x, with |mid| <= 2^-8 |x| and |lo| <= 2^-16 |x|.  The slices are
// those of three successive bf16 roundings; integer adds, masks, two subtractions and byte
// permutes only.  The slices of -x are the negated slices of x.
__device__ __forceinline__ uint32_t round_bf16_bits(uint32_t b) {
  return (b + 0x7fffu + ((b >> 16) & 1u)) & 0xffff0000u;
}
__device__ __forceinline__ void split_exact(float x, uint32_t& h, uint32_t& m, uint32_t& l) {
  h = round_bf16_bits(__float_as_uint(x));
  const float r = x - __uint_as_float(h);
  m = round_bf16_bits(__float_as_uint(r));
  l = __float_as_uint(r - __uint_as_float(m));
}
// Four values -> three slices, each packed as bf16 pairs in memory order.
__device__ __forceinline__ void split4_exact(float a, float b, float c, float d, uint2& hi, uint2& mid, uint2& lo) {
  uint32_t ha, ma, la, hb, mb, lb, hc, mc, lc, hd, md, ld;
  split_exact(a, ha, ma, la);
  split_exact(b, hb, mb, lb);
  split_exact(c, hc, mc, lc);
  split_exact(d, hd, md, ld);
  hi = make_uint2(__byte_perm(ha, hb, 0x7632), __byte_perm(hc, hd, 0x7632));
  mid = make_uint2(__byte_perm(ma, mb, 0x7632), __byte_perm(mc, md, 0x7632));
  lo = make_uint2(__byte_perm(la, lb, 0x7632), __byte_perm(lc, ld, 0x7632));
}
// Two values -> three packed slice words.
__device__ __forceinline__ void split2_exact(float a, float b, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  uint32_t ha, ma, la, hb, mb, lb;
  split_exact(a, ha, ma, la);
  split_exact(b, hb, mb, lb);
  hi = __byte_perm(ha, hb, 0x7632);
  mid = __byte_perm(ma, mb, 0x7632);
  lo = __byte_perm(la, lb, 0x7632);
}

}  // namespace tcx
