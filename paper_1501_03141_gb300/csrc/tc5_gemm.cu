// Blackwell (tcgen05) tensor-core kernel for the coefficients of the FP32
// projection term of the Sternheimer CG operator, sum_w sigma_w |w><w| x
// (Eq. stern with the occupied and deflated states w):
//
//   S[j][w] = sigma_w * sum_k P[w][k] X[bmap(j)][k]        (K = n_pw)
//
// in 3xTF32: every FP32 operand a is split into a_hi = tf32(a) and a_lo =
// tf32(a - a_hi), and a b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi, three
// tcgen05.mma.kind::tf32 per product with FP32 accumulation in tensor memory
// (a single TF32 product would perturb the CG operator at the 1e-4 level).
//
// Operands sit in shared memory in the K-major, no-swizzle layout of 8-row x
// 16-byte core matrices: core matrix (r / 8, k / 4) of a 32-wide K stage at
// (r / 8 * 8 + k / 4) * 128 bytes, so the leading (K) byte offset of the
// matrix descriptor is 128 and the stride (8-row) offset 1024.  Every K
// stage of 32 is accumulated into one of two tensor-memory accumulators and
// then added to FP32 registers (tcgen05.ld): measured over K = 6859 with
// cancelling sums, accumulating the whole K range in tensor memory left
// errors of 6.5e-7 of sum |terms| (rms), 30 times those of a sequential FP32
// FMA sum, while the flush after every stage gives 5e-9.
//
// A BF16 variant (PDEP_MIXED_BF16: the inner CG's coefficients to about
// 2^-8 relative) converts X and the states to BF16 and issues one
// tcgen05.mma.kind::f16 per 16-wide k-step; 16-bit core matrices hold 8 rows
// x 8 elements, so a 32-wide stage has 4 of them along K (stride 512 bytes).
//
// Every mbarrier wait is bounded (about a second of SM cycles); a wait that
// runs out marks the CTA aborted, the other warps give up their waits, the
// MMA-issuing thread waits (bounded) for its MMAs and copies in flight, the
// tensor memory is freed and DEV_TIMEOUT is set in the status word.
#include <algorithm>
#include <cstdint>

#include "linalg.cuh"
#include "profile.cuh"

namespace pdep {
namespace {

constexpr long long T5_WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// round to the nearest TF32 value, ties away from zero (the rounding of
// cvt.rna.tf32.f32), on the integer pipe, which measured 7% faster in the
// split: adding half a TF32 ulp to the magnitude bits and clearing the 13
// dropped mantissa bits carries into the exponent where it must; valid for
// all finite inputs
__device__ __forceinline__ uint32_t tf32_bits(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}
// float offset of element (row r, k) of a 32-wide K stage in the core-matrix
// layout: core matrix (r / 8, k / 4) at (r / 8 * 8 + k / 4) * 128 bytes,
// row r % 8 at 16 bytes, k % 4 at 4 bytes
__device__ __forceinline__ int cm_off(int r, int k) {
  return ((r >> 3) * 8 + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}
// shared-memory matrix descriptor, K-major, no swizzle: leading (K-direction)
// core-matrix stride 128 B, stride (8-row) 1024 B, sm_100-family version bit
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint64_t smem_desc_sbo(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | ((uint64_t)1 << 46);
}
// bf16 offset of element (row r, k) of a 32-wide stage in the 16-bit
// core-matrix layout (core (r / 8, k / 8) at (r / 8 * 4 + k / 8) * 128 bytes)
__device__ __forceinline__ int cm_off16(int r, int k) {
  return ((r >> 3) * 4 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(su32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}
// bounded wait for the phase of the given parity; false when it ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  const long long t0 = clock64();
  while (!mbar_try(bar, phase))
    if (clock64() - t0 > T5_WAIT_CYCLES) return false;
  return true;
}
// the same, giving up at once when another warp has aborted (and marking
// the abort when it runs out itself)
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t phase, volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try(bar, phase)) {
    if (*abort || clock64() - t0 > T5_WAIT_CYCLES) {
      *abort = 1;
      return false;
    }
  }
  return true;
}
// the same for warps whose wait is off the critical path: between polls the
// warp sleeps, leaving the issue slots of its SM sub-partition to the warps
// that share it
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t phase, volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try(bar, phase)) {
    if (*abort || clock64() - t0 > T5_WAIT_CYCLES) {
      *abort = 1;
      return false;
    }
    __nanosleep(200);
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
// bulk asynchronous global -> shared copy completing on an mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, int bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}
// 16 / 8 columns of the warp's 32 tensor-memory lanes; the wait carries the
// registers so that no use of them can be scheduled before it
__device__ __forceinline__ void tmem_ld16w(uint32_t taddr, float* out) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
                 "+r"(r[13]), "+r"(r[14]), "+r"(r[15])::"memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld8w(uint32_t taddr, float* out) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7])::"memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) out[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------------------
// Tile: 128 right-hand sides (tensor-memory lanes, MMA M) x NT states (MMA
// N; n_ext split into tiles of at most 128, padded to a multiple of 16), K
// in stages of 32.  The unit of work is one stage of one tile; the units
// (state tile, RHS tile, stage; stage fastest) are dealt out in equal
// contiguous ranges to one CTA per SM ("stream-K"); a CTA adds the sums of
// every tile it touches into S with atomics (S is zeroed first), so the load
// is balanced whatever the number of columns.
//
// The CTA's twelve warps work on different units at once and hand them on
// through mbarriers:
//   warps 0-2 (producers): cp.async of X rows (gathered through bmap,
//     zero-filled past N and K) into a ring of R raw FP32 slots, R - 1 units
//     ahead; then the split of unit i into hi and lo (elementwise: the slot
//     is already in the MMA layout) into converted buffer i % 2, once the
//     MMAs of unit i - 2 have released it;
//   warp 3, one lane: the unit's 12 MMAs (4 k-steps x 3 products) into
//     tensor-memory accumulator i % 2, committed to mbarriers, and the bulk
//     asynchronous copies of the states' pre-split hi / lo stage tiles
//     (tc5_split_states) into a ring of C5_PD slots;
//   warps 4-11 (flush): wait for unit i's accumulator, read it (warp w reads
//     lanes 32 (w % 4).. and half of the NT columns: one RHS row per
//     thread), release it and add it to FP32 registers; at the end of a tile
//     they scale by sigma_w and add into S.
// ---------------------------------------------------------------------------
constexpr int C5_THREADS = 384, C5_PD = 3, C5_NTMAX = 128, C5_RMAX = 6;
constexpr int C5_PROD = 96;                      // producer threads (warps 0-2)
constexpr int C5_SLOT = 128 * 32 * 4;            // one X stage (raw, hi or lo)
constexpr int C5_SMEM_MAX = 227 * 1024;          // opt-in shared memory per block
// one stage of the states: TF32 hi + lo (256 nt bytes) or BF16 (64 nt bytes)
__host__ __device__ inline int c5_pbytes(int nt, int bf = 0) { return bf ? 64 * nt : 256 * nt; }
// raw slots that fit beside the two converted buffers and the P ring
// (alignment slack and the static shared memory kept aside)
__host__ __device__ inline int c5_ring(int nt) {
  const int r = (C5_SMEM_MAX - 2048 - 4 * C5_SLOT - C5_PD * c5_pbytes(nt)) / C5_SLOT;
  return r < C5_RMAX ? r : C5_RMAX;
}
__host__ __device__ inline int c5_smem(int nt) {
  return (c5_ring(nt) + 4) * C5_SLOT + C5_PD * c5_pbytes(nt) + 1024;
}

struct C5Geom {
  int ntl, nt, nks;  // state tiles, states per tile (multiple of 16), K stages
};
__host__ __device__ inline C5Geom c5_geom(int n_ext, int K) {
  C5Geom g;
  g.ntl = (n_ext + C5_NTMAX - 1) / C5_NTMAX;
  const int per = (n_ext + g.ntl - 1) / g.ntl;
  g.nt = ((per + 15) / 16) * 16;
  g.nks = (K + 31) / 32;
  return g;
}
// position of a unit, advanced one unit at a time (no division in the loops)
struct C5Pos {
  int nt, rt, ks;
  __device__ __forceinline__ void next(const C5Geom& g, int rtiles) {
    if (++ks == g.nks) {
      ks = 0;
      if (++rt == rtiles) {
        rt = 0;
        ++nt;
      }
    }
  }
};

template <int BF>
__global__ void __launch_bounds__(C5_THREADS, 1)
    k_tc5_coeffs(int n_ext, int N, int K, C5Geom g, const unsigned char* __restrict__ Pt,
                 const float* __restrict__ X, long long ldx, const int* __restrict__ bmap,
                 const float* __restrict__ sigma, float* __restrict__ S, long long lds,
                 const int* __restrict__ ndev, unsigned* status) {
  extern __shared__ unsigned char c5_dyn[];
  // conv_full / conv_empty: converted buffer c holds unit i / is free again;
  // acc_full / acc_empty: accumulator a holds unit i / has been read;
  // p_full: P slot holds its stage
  __shared__ __align__(8) uint64_t conv_full[2], conv_empty[2], acc_full[2], acc_empty[2],
      p_full[C5_PD];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ volatile int prod_fail;
  if (ndev) N = min(N, *ndev);
  const int rtiles = (N + 127) / 128;
  const int U = g.ntl * rtiles * g.nks;
  const int u0 = (int)((long long)U * blockIdx.x / gridDim.x);
  const int n = (int)((long long)U * (blockIdx.x + 1) / gridDim.x) - u0;
  if (n <= 0) return;
  unsigned char* base = (unsigned char*)(((uintptr_t)c5_dyn + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = su32(base);
  const int R = c5_ring(g.nt);
  const uint32_t conv0 = sbase + R * C5_SLOT, p0 = conv0 + 4 * C5_SLOT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NT = g.nt;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"(256u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&conv_full[b])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&conv_empty[b])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&acc_full[b])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&acc_empty[b])), "r"(256));
    }
    for (int b = 0; b < C5_PD; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&p_full[b])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    prod_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  C5Pos start;
  start.ks = u0 % g.nks;
  start.rt = (u0 / g.nks) % rtiles;
  start.nt = u0 / g.nks / rtiles;

  if (warp < 3) {
    // ---------------- producers: X loads and the hi / lo split ----------------
    C5Pos ld = start;
    int ld_i = 0;
    auto issue = [&]() {  // cp.async of unit ld_i into raw slot ld_i % R; one group
      if (ld_i < n) {
        const uint32_t dst = sbase + (ld_i % R) * C5_SLOT;
        for (int e = tid; e < 128 * 8; e += C5_PROD) {
          const int r = e >> 3, c = e & 7;
          const int j = ld.rt * 128 + r, k = ld.ks * 32 + 4 * c;
          const int bytes = j < N ? max(0, min(16, 4 * (K - k))) : 0;
          const float* row = X + (long long)(j < N ? (bmap ? bmap[j] : j) : 0) * ldx;
          cp_async16(dst + 4 * cm_off(r, 4 * c),
                     bytes > 0 ? (const void*)(row + k) : (const void*)row, bytes);
        }
        ld.next(g, rtiles);
        ++ld_i;
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int q = 0; q < R - 1; ++q) issue();
    for (int i = 0; i < n; ++i) {
      issue();  // unit i + R - 1, into the slot unit i - 1 was split from
      // R - 1 groups may stay pending: the one of unit i has landed
      switch (R) {
        case 6: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      // converted buffer i % 2 was last read by the MMAs of unit i - 2
      if (tid == 0 && i >= 2 &&
          !mbar_wait_ab(&conv_empty[i & 1], (uint32_t)(((i >> 1) + 1) & 1), &abort_flag))
        prod_fail = 1;
      named_sync(1, C5_PROD);
      if (prod_fail) break;
      const float4* src = (const float4*)(base + (i % R) * C5_SLOT);
      uint4* hi = (uint4*)(base + R * C5_SLOT + (i & 1) * 2 * C5_SLOT);
      uint4* lo = hi + C5_SLOT / 16;
      if constexpr (BF) {
        // float4 f holds (r, k..k+3): f = (r / 8) 64 + (k / 4) 8 + r % 8
        unsigned char* b16 = (unsigned char*)hi;
        for (int f = tid; f < C5_SLOT / 16; f += C5_PROD) {
          const float4 v = src[f];
          const int r = (f >> 6) * 8 + (f & 7), k = ((f >> 3) & 7) * 4;
          *(uint2*)(b16 + 2 * cm_off16(r, k)) = make_uint2(bf16x2_bits(v.x, v.y), bf16x2_bits(v.z, v.w));
        }
      } else
      for (int f = tid; f < C5_SLOT / 16; f += C5_PROD) {
        const float4 v = src[f];
        uint4 h, l;
        h.x = tf32_bits(v.x);
        h.y = tf32_bits(v.y);
        h.z = tf32_bits(v.z);
        h.w = tf32_bits(v.w);
        l.x = tf32_bits(v.x - __uint_as_float(h.x));
        l.y = tf32_bits(v.y - __uint_as_float(h.y));
        l.z = tf32_bits(v.z - __uint_as_float(h.z));
        l.w = tf32_bits(v.w - __uint_as_float(h.w));
        hi[f] = h;
        lo[f] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      named_sync(1, C5_PROD);  // the split is complete; raw slot i % R is free
      if (tid == 0) mbar_arrive(&conv_full[i & 1]);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else if (warp == 3) {
    // ---------------- MMA issue and the states' bulk copies (one lane) ----------------
    if (lane == 0) {
      // D FP32; A, B TF32 (2) or BF16 (1); N = NT, M = 128
      const uint32_t fmt = BF ? 1u : 2u;
      const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      const int pb = c5_pbytes(NT, BF);
      C5Pos pp = start;
      int p_i = 0;
      auto issue_p = [&]() {
        if (p_i < n) {
          const unsigned char* src = Pt + (long long)(pp.nt * g.nks + pp.ks) * pb;
          bulk_g2s(p0 + (p_i % C5_PD) * pb, src, pb, &p_full[p_i % C5_PD]);
          pp.next(g, rtiles);
          ++p_i;
        }
      };
      for (int q = 0; q < C5_PD; ++q) issue_p();
      int mma_last = -1, p_used = -1;
      for (int i = 0; i < n; ++i) {
        if (!mbar_wait_ab(&conv_full[i & 1], (uint32_t)((i >> 1) & 1), &abort_flag)) break;
        if (!mbar_wait_ab(&p_full[i % C5_PD], (uint32_t)((i / C5_PD) & 1), &abort_flag)) break;
        p_used = i;
        // accumulator i % 2 was last read by the flush of unit i - 2
        if (i >= 2 &&
            !mbar_wait_ab(&acc_empty[i & 1], (uint32_t)(((i >> 1) + 1) & 1), &abort_flag))
          break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah0 = conv0 + (i & 1) * 2 * C5_SLOT, al0 = ah0 + C5_SLOT;
        const uint32_t bh0 = p0 + (i % C5_PD) * pb, bl0 = bh0 + NT * 128;
        const uint32_t td = tmem + (uint32_t)((i & 1) * 128);
        if constexpr (BF) {
          // two k-steps of 16 (2 core matrices along K each), one product
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const uint64_t ad = smem_desc_sbo(ah0 + s * 256, 512), bd = smem_desc_sbo(bh0 + s * 256, 512);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(td),
                "l"(ad), "l"(bd), "r"(idesc), "r"(s > 0 ? 1u : 0u)
                : "memory");
          }
        } else
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint32_t off = s * 256;  // 8 k = 2 core matrices along K
          const uint64_t ah = smem_desc(ah0 + off), al = smem_desc(al0 + off);
          const uint64_t bh = smem_desc(bh0 + off), bl = smem_desc(bl0 + off);
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(td),
              "l"(al), "l"(bh), "r"(idesc), "r"(s > 0 ? 1u : 0u)
              : "memory");
          asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(td), "l"(ah),
                       "l"(bl), "r"(idesc)
                       : "memory");
          asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(td), "l"(ah),
                       "l"(bh), "r"(idesc)
                       : "memory");
        }
        mma_commit(&acc_full[i & 1]);
        mma_commit(&conv_empty[i & 1]);
        mma_last = i;
        // P of unit i + C5_PD - 1 goes to unit i - 1's slot, free once its MMAs end
        if (p_i < n && i >= 1) {
          if (!mbar_wait_ab(&acc_full[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), &abort_flag))
            break;
          issue_p();
        }
      }
      if (abort_flag) {
        // MMAs complete in order: the last one's commit covers them all; the
        // bulk copies issued but not consumed must land too (bounded waits)
        if (mma_last >= 0) mbar_wait(&acc_full[mma_last & 1], (uint32_t)((mma_last >> 1) & 1));
        for (int u = p_used + 1; u < p_i; ++u)
          mbar_wait(&p_full[u % C5_PD], (uint32_t)((u / C5_PD) & 1));
      }
    }
  } else {
    // ---------------- flush: accumulators into registers, tiles into S ----------------
    constexpr int HMAX = C5_NTMAX / 2;
    const int half = NT / 2, ch = ((warp - 4) >> 2) * half;  // this warp's columns
    float acc[HMAX];
#pragma unroll
    for (int c = 0; c < HMAX; ++c) acc[c] = 0.f;
    C5Pos fp = start;
    const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
    for (int i = 0; i < n; ++i) {
      const bool ok = __all_sync(
          0xffffffffu, mbar_wait_sleep(&acc_full[i & 1], (uint32_t)((i >> 1) & 1), &abort_flag));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ta = tmem + lane_addr + (uint32_t)((i & 1) * 128 + ch);
#pragma unroll
      for (int c16 = 0; c16 < HMAX / 16; ++c16) {
        float v[16];
        if (16 * c16 + 16 <= half) {
          tmem_ld16w(ta + 16 * c16, v);
#pragma unroll
          for (int e = 0; e < 16; ++e) acc[16 * c16 + e] += v[e];
        } else if (16 * c16 + 8 <= half) {
          tmem_ld8w(ta + 16 * c16, v);
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[16 * c16 + e] += v[e];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acc_empty[i & 1]);
      if (i == n - 1 || fp.ks == g.nks - 1) {
        // this CTA's sums of the tile: scale by sigma_w and add into S
        const int j = fp.rt * 128 + 32 * (warp & 3) + lane;
        const int w0 = fp.nt * NT + ch;
        if (j < N) {
          float* srow = S + (long long)j * lds;
#pragma unroll
          for (int c4 = 0; c4 < HMAX / 4; ++c4)
            if (4 * c4 < half) {
              const int w = w0 + 4 * c4;
              if (w + 3 < n_ext) {
                const float4 sg = *(const float4*)(sigma + w);
                atomicAdd((float4*)(srow + w),
                          make_float4(sg.x * acc[4 * c4], sg.y * acc[4 * c4 + 1],
                                      sg.z * acc[4 * c4 + 2], sg.w * acc[4 * c4 + 3]));
              } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  if (w + e < n_ext) atomicAdd(srow + w + e, sigma[w + e] * acc[4 * c4 + e]);
              }
            }
        }
#pragma unroll
        for (int c = 0; c < HMAX; ++c) acc[c] = 0.f;
      }
      fp.next(g, rtiles);
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(status, (unsigned)DEV_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
}

// states P[w][k] (w < n_ext, k < K, row stride ldp) -> hi / lo tiles
// [state tile][stage][hi | lo][NT x 32 core-matrix layout], zero-padded
__global__ void k_tc5_split(int n_ext, int K, C5Geom g, const float* __restrict__ P, long long ldp,
                            float* __restrict__ Pt) {
  const long long per = 32LL * g.nt;
  const long long total = (long long)g.ntl * g.nks * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / per;
    const int rem = (int)(e % per), r = rem >> 5, k = rem & 31;
    const int nt = (int)(blk / g.nks), ks = (int)(blk % g.nks);
    const int w = nt * g.nt + r, kk = ks * 32 + k;
    const float x = (w < n_ext && kk < K) ? P[(long long)w * ldp + kk] : 0.f;
    const uint32_t h = tf32_bits(x);
    float* out = Pt + blk * 2 * per;
    out[cm_off(r, k)] = __uint_as_float(h);
    out[per + cm_off(r, k)] = __uint_as_float(tf32_bits(x - __uint_as_float(h)));
  }
}

// states -> BF16 tiles [state tile][stage][NT x 32 16-bit core-matrix layout]
__global__ void k_tc5_split_bf16(int n_ext, int K, C5Geom g, const float* __restrict__ P,
                                 long long ldp, unsigned short* __restrict__ Pt) {
  const long long per = 32LL * g.nt;
  const long long total = (long long)g.ntl * g.nks * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / per;
    const int rem = (int)(e % per), r = rem >> 5, k = rem & 31;
    const int nt = (int)(blk / g.nks), ks = (int)(blk % g.nks);
    const int w = nt * g.nt + r, kk = ks * 32 + k;
    const float x = (w < n_ext && kk < K) ? P[(long long)w * ldp + kk] : 0.f;
    Pt[blk * per + cm_off16(r, k)] = (unsigned short)(bf16x2_bits(x, 0.f) & 0xFFFFu);
  }
}

int t5_sms() {
  static const int n = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 152;
  }();
  return n;
}

}  // namespace

size_t tc5_split_floats(int n_ext, int K) {
  if (n_ext <= 0 || K <= 0) return 0;
  const C5Geom g = c5_geom(n_ext, K);
  return (size_t)g.ntl * g.nks * 64 * g.nt;
}

cudaError_t tc5_split_states(int n_ext, int K, const float* P, long long ldp, float* Pt,
                             cudaStream_t st) {
  if (n_ext <= 0 || K <= 0) return cudaSuccess;
  const C5Geom g = c5_geom(n_ext, K);
  const long long total = (long long)g.ntl * g.nks * 32 * g.nt;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * t5_sms());
  count_launch();
  k_tc5_split<<<blocks, 256, 0, st>>>(n_ext, K, g, P, ldp, Pt);
  return cudaGetLastError();
}

size_t tc5_split_bytes_bf16(int n_ext, int K) {
  if (n_ext <= 0 || K <= 0) return 0;
  const C5Geom g = c5_geom(n_ext, K);
  return (size_t)g.ntl * g.nks * c5_pbytes(g.nt, 1);
}

cudaError_t tc5_split_states_bf16(int n_ext, int K, const float* P, long long ldp, void* Pt,
                                  cudaStream_t st) {
  if (n_ext <= 0 || K <= 0) return cudaSuccess;
  const C5Geom g = c5_geom(n_ext, K);
  const long long total = (long long)g.ntl * g.nks * 32 * g.nt;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * t5_sms());
  count_launch();
  k_tc5_split_bf16<<<blocks, 256, 0, st>>>(n_ext, K, g, P, ldp, (unsigned short*)Pt);
  return cudaGetLastError();
}

cudaError_t tc5_proj_coeffs(int n_ext, int N, int K, const void* Pt, const float* X,
                            long long ldx, const int* bmap, const float* sigma, float* S,
                            long long lds, cudaStream_t st, const int* ndev, unsigned* status,
                            bool bf16) {
  if (n_ext <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0) return cudaMemsetAsync(S, 0, sizeof(float) * (size_t)lds * N, st);
  const C5Geom g = c5_geom(n_ext, K);
  const int smem = c5_smem(g.nt);
  static int attr[2] = {0, 0};
  if (smem > attr[bf16]) {
    cudaError_t e = cudaFuncSetAttribute(bf16 ? k_tc5_coeffs<1> : k_tc5_coeffs<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr[bf16] = smem;
  }
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(float) * (size_t)lds * N, st);
  if (e != cudaSuccess) return e;
  // one CTA per SM, at least four units each
  const long long units = (long long)g.ntl * ((N + 127) / 128) * g.nks;
  if (units > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)std::max<long long>(1, std::min<long long>(t5_sms(), units / 4));
  ProfScope ps(PC_GEMM_TF32, st, 2.0 * n_ext * N * (double)K,
               ((double)n_ext * K + (double)K * N + (double)n_ext * N) * sizeof(float), ndev, N);
  count_launch();
  const unsigned char* pt = (const unsigned char*)Pt;
  if (bf16)
    k_tc5_coeffs<1><<<grid, C5_THREADS, smem, st>>>(n_ext, N, K, g, pt, X, ldx, bmap, sigma, S,
                                                    lds, ndev, status);
  else
    k_tc5_coeffs<0><<<grid, C5_THREADS, smem, st>>>(n_ext, N, K, g, pt, X, ldx, bmap, sigma, S,
                                                    lds, ndev, status);
  return cudaGetLastError();
}

}  // namespace pdep
