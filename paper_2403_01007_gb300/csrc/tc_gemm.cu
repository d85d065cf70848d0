// tcgen05 BF16 GEMM with TMA loads and TMEM accumulators (sm_103a).
//
// A persistent CTA (one per SM) walks a list of work items, each a 128 x 256
// FP32 tile of A * B^T (both operands K-major BF16 in global memory, padded to
// whole tiles) over a range of K blocks (a split index selects the range when
// K is split), and writes alpha * tile into an FP64 output through a strided
// multi-level view (overwrite or accumulate), so that permuted tensor layouts
// need no separate copy. TMEM holds two accumulators: the epilogue of one item
// overlaps the MMAs of the next, and the set-up (TMEM allocation, barriers,
// pipeline fill) is paid once per CTA instead of once per tile. Warp roles:
//   warp 4    : TMA producer, 4-stage ring of (A 128x64, B 256x64) tiles,
//               128-byte swizzle, completion on mbarriers (expect_tx)
//   warp 5    : one elected thread issues tcgen05.mma.kind::f16 (M=128,
//               N=256, K=16 per instruction, 4 per stage) into accumulator
//               (item & 1), commits each stage back to the producer and the
//               finished accumulator to the epilogue; before reusing an
//               accumulator it waits until the epilogue has read it
//   warps 0-3 : epilogue, tcgen05.ld 32 lanes x 32 columns at a time; when
//               the output's row index is the unit-stride one each thread
//               stores its own row (consecutive lanes, consecutive
//               addresses), otherwise the block is transposed through shared
//               memory so that lanes walk the columns
// Every mbarrier wait is bounded; on expiry the kernel records an error code
// and the remaining roles skip their work, so a fault in the pipeline shows
// up as an error status instead of a hang. TMEM is always freed.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <stdexcept>
#include <string>

#include "backend.h"
#include "tc_gemm.h"

namespace sccsd {

void count_launch();

namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
// dynamic shared memory of the kernel with NST pipeline stages and EW epilogue warps
constexpr int smem_bytes(int NST, int EW) {
  return 1024 /*align slack*/ + NST * STAGE_BYTES + 256 /*barriers*/ + EW * 32 * 33 * 4 +
         2 * EW * 32 * 8 /*row and column offsets*/;
}
constexpr int TMEM_COLS = 512;  // two 128 x 256 FP32 accumulators
constexpr uint32_t WAIT_LIMIT = 1u << 24;  // polls before a wait is declared failed

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
      " selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false (and records code) when the limit is reached
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
  for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (i > 32) __nanosleep(64);
  }
  atomicCAS(err, 0, code);
  return false;
}

__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)(16u >> 4) << 16;           // leading byte offset (unused, K-major SW128)
  d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version (tcgen05)
  d |= (uint64_t)2 << 61;                    // 128-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: BF16 x BF16 -> FP32, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4)                      // D format FP32
         | (1u << 7)                    // A format BF16
         | (1u << 10)                   // B format BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ int64_t level_offset(int n, const int64_t* e, const int64_t* s,
                                                int64_t i) {
  int64_t off = 0;
  for (int l = n - 1; l > 0; --l) {
    off += (i % e[l]) * s[l];
    i /= e[l];
  }
  return off + i * s[0];
}
__device__ __forceinline__ int64_t out_row(const OutView& v, int64_t r) {
  return level_offset(v.nr, v.re, v.rs, r);
}
__device__ __forceinline__ int64_t out_col(const OutView& v, int64_t c) {
  return level_offset(v.nc, v.ce, v.cs, c);
}

// Work items are (split z, N tile, M tile), M fastest (nfast = 0) or N fastest
// (nfast = 1); a persistent CTA takes items blockIdx.x, blockIdx.x + gridDim.x,
// ... so that the CTAs working at one time share the tile of the operand
// that is expensive to re-read (read once from HBM, then served from L2).
struct TcItem {
  int64_t m0, n0;
  int z;
};
__device__ __forceinline__ TcItem tc_item(int64_t w, int64_t mt, int64_t nt, int nfast) {
  TcItem r;
  const int64_t inner = nfast ? nt : mt, outer = nfast ? mt : nt;
  const int64_t a = w % inner, rest = w / inner;
  const int64_t b = rest % outer;
  r.m0 = (nfast ? b : a) * BM;
  r.n0 = (nfast ? a : b) * BN;
  r.z = (int)(rest / outer);
  return r;
}

__device__ __forceinline__ bool bf16_positive(uint16_t u) { return (u & 0x8000u) == 0 && u != 0; }

// Epilogue of one 32-column chunk of a learned-part layer (MODE = MlpMode):
// thread `lane` of the warp holds row `row` of the tile, columns cb .. cb + 31
// in r. Rows past M write only zeros into the transposed output, so that a
// later contraction over rows reads zeros there.
template <int MODE>
__device__ __forceinline__ void mlp_chunk(const MlpEpi& e, int64_t row, int64_t M, int64_t cb,
                                          int64_t N, int z, int64_t split_stride,
                                          const uint32_t* r) {
  if constexpr (MODE == MLP_HIDDEN || MODE == MLP_RELU_BACK) {
    const bool rv = row < M;
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const int64_t c0 = cb + j, c1 = cb + j + 1;
      float x0 = __uint_as_float(r[j]), x1 = __uint_as_float(r[j + 1]);
      if constexpr (MODE == MLP_HIDDEN) {
        x0 = c0 < N ? fmaxf(x0 + e.bias[c0], 0.f) : 0.f;
        x1 = c1 < N ? fmaxf(x1 + e.bias[c1], 0.f) : 0.f;
      } else {
        x0 = (rv && c0 < N && bf16_positive(e.maskT[c0 * e.ldm + row])) ? x0 : 0.f;
        x1 = (rv && c1 < N && bf16_positive(e.maskT[c1 * e.ldm + row])) ? x1 : 0.f;
      }
      if (!rv) x0 = x1 = 0.f;
      __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
      pk[j / 2] = *reinterpret_cast<const uint32_t*>(&h);
      if (e.outT) {
        if (c0 < N) e.outT[c0 * e.ldt + row] = (uint16_t)(pk[j / 2] & 0xFFFFu);
        if (c1 < N) e.outT[c1 * e.ldt + row] = (uint16_t)(pk[j / 2] >> 16);
      }
    }
    if (rv && e.out) {
      uint4* dst = reinterpret_cast<uint4*>(e.out + row * e.ldo + cb);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        dst[k] = make_uint4(pk[4 * k], pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
    }
  } else if constexpr (MODE == MLP_OUTPUT) {
    if (row >= M) return;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (cb + j < N) e.outf[row * e.ldf + cb + j] = __uint_as_float(r[j]) + e.bias[cb + j];
  } else {
    if (row >= M) return;
    float* p = e.outf + (int64_t)z * split_stride + row * e.ldf;
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (cb + j < N) p[cb + j] = __uint_as_float(r[j]);
  }
}

// NST pipeline stages; EW = 4 or 8 epilogue warps (with 8, two groups of four
// each own one TMEM accumulator and take alternate items: more stores in
// flight for the epilogue-bound short-K contractions). MODE 0 writes FP64
// through the output view; MODE 1..4 are the learned part's epilogues.
template <int NST, int EW, int MODE = 0>
__global__ void __launch_bounds__((EW + 2) * 32, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int64_t M, int64_t N, int64_t mt, int64_t nt, int nfast, int64_t items, int nk_total,
              int kbs,
              double alpha, double* __restrict__ C, int64_t split_stride, const OutView ov,
              int accumulate, int* err, const MlpEpi mep) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  constexpr int STAGES = NST;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // [2]: accumulator buffer ready for the epilogue
  uint64_t* acc_empty = acc_full + 2;    // [2]: epilogue done reading the buffer
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  float* epi = (float*)(smem + STAGES * STAGE_BYTES + 256);
  int64_t* row_off = (int64_t*)(epi + EW * 32 * 33);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // K blocks of split z: [z * kbs, z * kbs + nk(z))
  auto nk_of = [&](int z) { return (nk_total - z * kbs < kbs) ? nk_total - z * kbs : kbs; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&acc_empty[b])));
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == EW) {
    if (lane == 0) {
      // TMA producer over all items of this CTA; g counts k-blocks globally
      int64_t issued_last[STAGES];
      for (int s = 0; s < STAGES; ++s) issued_last[s] = -1;
      int64_t g = 0;
      for (int64_t w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        const TcItem it = tc_item(w, mt, nt, nfast);
        const int nk = nk_of(it.z), kb0 = it.z * kbs;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % STAGES);
          if (g >= STAGES) {
            if (!mbar_wait(smem_u32(&empty[s]), (uint32_t)((g / STAGES) - 1) & 1, err, 1)) {
              *abort_flag = 1;
              break;
            }
          }
          if (*abort_flag) break;
          const uint32_t fb = smem_u32(&full[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                       "r"(STAGE_BYTES)
                       : "memory");
          const int x = (kb0 + kb) * BK;
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(sA + s * A_BYTES)),
              "l"((uint64_t)&tmA), "r"(fb), "r"(x), "r"((int)it.m0)
              : "memory");
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(sB + s * B_BYTES)),
              "l"((uint64_t)&tmB), "r"(fb), "r"(x), "r"((int)it.n0)
              : "memory");
          issued_last[s] = g;
        }
      }
      // make sure no copy issued by this CTA is still in flight at exit
      for (int s = 0; s < STAGES; ++s)
        if (issued_last[s] >= 0)
          mbar_wait(smem_u32(&full[s]), (uint32_t)(issued_last[s] / STAGES) & 1, err, 2);
    }
  } else if (warp == EW + 1) {
    if (lane == 0) {
      // MMA issuer: item number i of this CTA accumulates in TMEM buffer i & 1
      constexpr uint32_t idesc = make_idesc(BM, BN);
      int64_t g = 0;
      int64_t i = 0;
      for (int64_t w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, ++i) {
        const TcItem it = tc_item(w, mt, nt, nfast);
        const int nk = nk_of(it.z);
        const int b = (int)(i & 1);
        if (i >= 2) {
          // the epilogue has read this buffer's previous tile
          if (!mbar_wait(smem_u32(&acc_empty[b]), (uint32_t)((i / 2) - 1) & 1, err, 5)) {
            *abort_flag = 1;
            break;
          }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dst = tmem + (uint32_t)(b * BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb, ++g) {
          const int s = (int)(g % STAGES);
          if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(g / STAGES) & 1, err, 3) || *abort_flag) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t ad = make_desc_sw128(a0 + k * 32);
            const uint64_t bd = make_desc_sw128(b0 + k * 32);
            const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(&empty[s]))
              : "memory");
        }
        // accumulator of this item ready (or the pipeline was abandoned)
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&acc_full[b]))
            : "memory");
        if (!ok) break;
      }
    }
  } else {
    // epilogue warp: TMEM lanes 32*q .. 32*q+31 of the items of its group
    constexpr int G = EW / 4;            // groups of four warps
    // old values of an accumulating store read ahead in batches of OLDN
    // (fewer registers with eight epilogue warps)
    constexpr int OLDN = EW == 8 ? 8 : 32;
    const int q = warp % 4, grp = warp / 4;
    float* buf = epi + warp * 32 * 33;
    int64_t* roff = row_off + warp * 32;
    int64_t* coff = row_off + EW * 32 + warp * 32;
    int64_t i = grp;
    const bool rows_fast = ov.rs[ov.nr - 1] == 1 && ov.cs[ov.nc - 1] != 1;
    for (int64_t w = blockIdx.x + (int64_t)grp * gridDim.x; w < items;
         w += (int64_t)G * gridDim.x, i += G) {
      if (*abort_flag) break;
      const TcItem it = tc_item(w, mt, nt, nfast);
      const int b = (int)(i & 1);
      const bool ok = mbar_wait(smem_u32(&acc_full[b]), (uint32_t)(i / 2) & 1, err, 4);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok || *abort_flag) {
        *abort_flag = 1;
        break;
      }
      if constexpr (MODE == 0) {
        const int64_t row = it.m0 + q * 32 + lane;
        roff[lane] = row < M ? out_row(ov, row) : -1;
      }
      __syncwarp();
      double* Cz = C + (int64_t)it.z * split_stride;
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (it.n0 + c0 >= N) break;  // warp-uniform: no valid column left
        uint32_t r[32];
        const uint32_t taddr =
            tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
            "[%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
              "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
              "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
              "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if constexpr (MODE != 0) {
          mlp_chunk<MODE>(mep, it.m0 + q * 32 + lane, M, it.n0 + c0, N, it.z, split_stride, r);
          continue;
        }
        {
          // output offsets of this chunk's 32 columns, one per lane
          const int64_t col = it.n0 + c0 + lane;
          coff[lane] = col < N ? out_col(ov, col) : -1;
        }
        __syncwarp();
        // Accumulation reads all 32 old values of a thread before the first
        // store, so that the loads overlap instead of each waiting on HBM.
        if (rows_fast) {
          // lane = row: for each column the warp stores 32 consecutive rows
          const int64_t ro = roff[lane];
#pragma unroll
          for (int h = 0; h < 32; h += OLDN) {
            double old[OLDN];
#pragma unroll
            for (int j = 0; j < OLDN; ++j) {
              const int64_t co = coff[h + j];
              old[j] = (accumulate && ro >= 0 && co >= 0) ? Cz[ro + co] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < OLDN; ++j) {
              const int64_t co = coff[h + j];
              if (ro >= 0 && co >= 0)
                Cz[ro + co] = old[j] + alpha * (double)__uint_as_float(r[h + j]);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) buf[lane * 33 + j] = __uint_as_float(r[j]);
          __syncwarp();
          const int64_t co = coff[lane];
#pragma unroll
          for (int h = 0; h < 32; h += OLDN) {
            double old[OLDN];
#pragma unroll
            for (int j = 0; j < OLDN; ++j) {
              const int64_t ro = roff[h + j];
              old[j] = (accumulate && ro >= 0 && co >= 0) ? Cz[ro + co] : 0.0;
            }
#pragma unroll
            for (int j = 0; j < OLDN; ++j) {
              const int64_t ro = roff[h + j];
              if (ro >= 0 && co >= 0)
                Cz[ro + co] = old[j] + alpha * (double)buf[(h + j) * 33 + lane];
            }
          }
        }
        __syncwarp();  // buf and coff are rewritten by the next chunk
      }
      // this warp has read its lanes of buffer b: hand it back to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b]))
                     : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

// x = sum_s slice_s with slice_s = bf16(x - sum_{r<s} slice_r); K padded with
// zeros (padding rows are not written: their products are never stored). The
// source is a strided view; a 32 x 64 tile goes through shared memory so that
// reads walk the source's unit-stride index and writes walk k.
__device__ __forceinline__ int64_t vrow(const MatView& v, int64_t r) {
  return v.n2r ? (r / v.n2r) * v.sr1 + (r % v.n2r) * v.sr2 : r * v.sr2;
}
__device__ __forceinline__ int64_t vk(const MatView& v, int64_t k) {
  return v.n2k ? (k / v.n2k) * v.sk1 + (k % v.n2k) * v.sk2 : k * v.sk2;
}

constexpr int CR = 64, CK = 64;  // conversion tile: rows x K

__global__ void __launch_bounds__(256, 3)
    k_split_bf16_view(MatView X, int64_t rows, int64_t K, int64_t rows_pad, int64_t k_pad,
                      int slices, __nv_bfloat16* __restrict__ out) {
  __shared__ double tile[CR][CK + 1];
  __shared__ int64_t roff[CR], koff[CK];
  const int64_t ktiles = k_pad / CK;
  const int64_t tiles = (rows_pad / CR) * ktiles;
  const bool kfast = X.sk2 == 1;
  const int64_t sstride = rows_pad * k_pad;
  const int tid = threadIdx.x;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t r0 = (t / ktiles) * CR, k0 = (t % ktiles) * CK;
    // rows beyond `rows` only feed products that are never stored: left as is
    if (r0 >= rows) continue;
    // view offsets of the tile's rows and K indices, once per tile
    if (tid < CR) {
      const int64_t r = r0 + tid;
      roff[tid] = r < rows ? vrow(X, r) : -1;
    } else if (tid < CR + CK) {
      const int64_t k = k0 + tid - CR;
      koff[tid - CR] = k < K ? vk(X, k) : -1;
    }
    __syncthreads();
    // all 16 loads of a thread in flight before the first shared-memory store;
    // consecutive lanes walk the source's unit-stride index
    double val[CR * CK / 256];
#pragma unroll
    for (int q = 0; q < CR * CK / 256; ++q) {
      const int e = tid + 256 * q;
      const int rr = kfast ? e / CK : e % CR;
      const int kk = kfast ? e % CK : e / CR;
      const int64_t ro = roff[rr], ko = koff[kk];
      val[q] = (ro >= 0 && ko >= 0) ? __ldg(X.p + ro + ko) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < CR * CK / 256; ++q) {
      const int e = tid + 256 * q;
      const int rr = kfast ? e / CK : e % CR;
      const int kk = kfast ? e % CK : e / CR;
      tile[rr][kk] = val[q];
    }
    __syncthreads();
    // a warp writes one row's 64 K values as 32 bf16x2 (128 bytes)
#pragma unroll
    for (int q = 0; q < CR * CK / 512; ++q) {
      const int e = tid + 256 * q;
      const int rr = e / (CK / 2), kk = 2 * (e % (CK / 2));
      if (r0 + rr >= rows) continue;
      double x0 = tile[rr][kk], x1 = tile[rr][kk + 1];
      const int64_t o = (r0 + rr) * k_pad + k0 + kk;
      for (int s = 0; s < slices; ++s) {
        __nv_bfloat162 b;
        b.x = __double2bfloat16(x0);
        b.y = __double2bfloat16(x1);
        *reinterpret_cast<__nv_bfloat162*>(out + s * sstride + o) = b;
        x0 -= (double)__bfloat162float(b.x);
        x1 -= (double)__bfloat162float(b.y);
      }
    }
    __syncthreads();
  }
}

// C (= or +=) sum_z part[z] through the output view (split-K reduction; the
// partials already carry alpha)
__global__ void k_sum_splits(int64_t M, int64_t N, int splits, const double* __restrict__ part,
                             double* __restrict__ C, const OutView ov, int accumulate) {
  const int64_t n = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * n + e];
    double* p = C + out_row(ov, e / N) + out_col(ov, e % N);
    *p = accumulate ? *p + s : s;
  }
}

// ------------------------------------------------------------------ ladder build
//
// The particle-particle ladder of the T1-transformed Hamiltonian (Sec. 2.4.2)
// contracts the amplitudes with the vvvv integrals g_acbd = sum_J L^J_ac L^J_bd
// of the Cholesky vectors. They are never stored: for each pair (a, b), a <= b,
// of a chunk this kernel forms the v x v block W[c][d] = g_acbd on the tensor
// cores (M = c, N = d, K = J; A = the rows (a, c) and B = the rows (b, d) of the
// operand Lt[(p, q)][J] = L^J_pq over the virtual block) and writes
//   G+[pair][q(c, d)] = W[c][d] + W[d][c],   G-[pair][q(c, d)] = W[c][d] - W[d][c]
// for c <= d (q the packed index c*v - c(c-1)/2 + d - c) as BF16 slices of two
// K-major operands of the contraction kernel above. The symmetric and
// antisymmetric combinations halve the contraction twice over (pairs a <= b
// and c <= d), and W[d][c] comes from the same block, so each g_acbd is
// computed once per unordered pair (ac) <-> (bd), up to the diagonal blocks.
// Rows c < 128 and c >= 128 (v > 128) are two halves with their own TMEM
// accumulators (columns 0 .. and 256 ..), computed one after the other, so
// that the epilogue of one half overlaps the MMAs of the next.
// Warp roles:
//   warp 16   : TMA producer; one stage = A rows a*v + 128 h .. + 127 and B
//               rows b*v .. b*v + NB - 1 of one 64-wide K block; slice
//               products (0,0), (0,1), (1,0) in turn
//   warp 17   : one elected thread issues the MMAs of each half into its
//               accumulator, N = NB = v rounded up to 16
//   warps 0-15: epilogue; warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows c)
//               and the column chunks ch with ch % 4 = w / 4. Phase 1 writes the
//               upper triangle W[c][d], d > c, to shared memory (FP32); phase
//               2 takes the lower triangle from TMEM, forms both combinations
//               with the stored transpose and packs them in place as BF16
//               pairs (the second slice, when there is one, goes straight to
//               global memory); once both halves are done the packed
//               triangle is streamed out with 16-byte loads and 8-byte
//               stores, while the MMAs of the next pair already run.
// Every mbarrier wait is bounded as in k_tc_gemm; the epilogue warps meet at
// named barriers on every path, so an abort never leaves one of them waiting.
constexpr int LB_EPI = 16;                     // epilogue warps (four per TMEM lane quadrant)
constexpr int LB_THREADS = (LB_EPI + 2) * 32;

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
      "[%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(LB_EPI * 32) : "memory");
}

// HS (one BF16 slice): the upper triangle is kept as BF16, which leaves room
// for a fourth pipeline stage; phase 2 rewrites G+ in place and stores G- to
// global memory at once. Otherwise (two slices) it is kept in FP32 and phase 2
// packs G+ and G- in place.
template <bool HS>
__global__ void __launch_bounds__(LB_THREADS, 1)
    k_ladder_build(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int v, int NB, int two, int nkb, int nprod, int64_t slice_rows, int stages,
                   const int* __restrict__ pairs, int64_t p_begin, int64_t npairs,
                   __nv_bfloat16* __restrict__ gp, __nv_bfloat16* __restrict__ gm,
                   int64_t out_ld, int64_t out_sstride, int nsl, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int stage_bytes = A_BYTES + NB * BK * 2;
  uint64_t* full = (uint64_t*)(smem + stages * stage_bytes);
  uint64_t* empty = full + stages;
  uint64_t* acc_full = empty + stages;   // [2], one per half
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  float* S = (float*)(smem + stages * stage_bytes + 256);
  uint32_t* Su = (uint32_t*)S;
  __nv_bfloat16* Sh = (__nv_bfloat16*)S;
  const int64_t Pv = (int64_t)v * (v + 1) / 2;
  const int64_t P4 = (Pv + 3) / 4;
  const int H = two ? 2 : 1;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    for (int h = 0; h < 2; ++h) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[h])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acc_empty[h])),
                   "n"(LB_EPI));
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the padding of the last group of four entries reads as zero in phase 3
  const int64_t P8 = (Pv + 7) / 8;
  if (HS) {
    if (threadIdx.x < 8 && Pv + threadIdx.x < 8 * P8) Sh[Pv + threadIdx.x] = __float2bfloat16(0.0f);
  } else {
    if (threadIdx.x < 4 && Pv + threadIdx.x < 4 * P4) Su[Pv + threadIdx.x] = 0u;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == LB_EPI) {
    if (lane == 0) {
      int64_t issued_last[8];
      for (int s = 0; s < 8; ++s) issued_last[s] = -1;
      int64_t g = 0;
      for (int64_t w = blockIdx.x; w < npairs && !*abort_flag; w += gridDim.x) {
        const int ab = __ldg(pairs + p_begin + w);
        const int a = ab >> 16, b = ab & 0xffff;
        for (int h = 0; h < H && !*abort_flag; ++h) {
          for (int pr = 0; pr < nprod && !*abort_flag; ++pr) {
            const int sa = pr == 2 ? 1 : 0, sb = pr == 1 ? 1 : 0;
            const int ra = (int)(sa * slice_rows) + a * v + h * BM;
            const int rb = (int)(sb * slice_rows) + b * v;
            for (int kb = 0; kb < nkb; ++kb, ++g) {
              const int s = (int)(g % stages);
              if (g >= stages) {
                if (!mbar_wait(smem_u32(&empty[s]), (uint32_t)((g / stages) - 1) & 1, err, 11)) {
                  *abort_flag = 1;
                  break;
                }
              }
              if (*abort_flag) break;
              const uint32_t fb = smem_u32(&full[s]);
              asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                           "r"(stage_bytes)
                           : "memory");
              uint8_t* st = smem + (size_t)s * stage_bytes;
              const int x = kb * BK;
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                  " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(st)),
                  "l"((uint64_t)&tmA), "r"(fb), "r"(x), "r"(ra)
                  : "memory");
              asm volatile(
                  "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                  " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(st + A_BYTES)),
                  "l"((uint64_t)&tmB), "r"(fb), "r"(x), "r"(rb)
                  : "memory");
              issued_last[s] = g;
            }
          }
        }
      }
      for (int s = 0; s < stages; ++s)
        if (issued_last[s] >= 0)
          mbar_wait(smem_u32(&full[s]), (uint32_t)(issued_last[s] / stages) & 1, err, 12);
    }
  } else if (warp == LB_EPI + 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(BM, NB);
      int64_t g = 0, i = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < npairs && ok && !*abort_flag; w += gridDim.x, ++i) {
        for (int h = 0; h < H && ok; ++h) {
          if (i >= 1) {
            // the epilogue has read this half's accumulator of the previous pair
            if (!mbar_wait(smem_u32(&acc_empty[h]), (uint32_t)((i - 1) & 1), err, 15)) {
              *abort_flag = 1;
              ok = false;
              break;
            }
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dst = tmem + (uint32_t)(h * BN);
          for (int pr = 0; pr < nprod && ok; ++pr) {
            for (int kb = 0; kb < nkb; ++kb, ++g) {
              const int s = (int)(g % stages);
              if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(g / stages) & 1, err, 13) ||
                  *abort_flag) {
                *abort_flag = 1;
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              uint8_t* st = smem + (size_t)s * stage_bytes;
              const uint32_t a0 = smem_u32(st), b0 = smem_u32(st + A_BYTES);
#pragma unroll
              for (int k = 0; k < BK / 16; ++k) {
                const uint64_t ad = make_desc_sw128(a0 + k * 32);
                const uint64_t bd = make_desc_sw128(b0 + k * 32);
                const uint32_t acc = (pr > 0 || kb > 0 || k > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
              }
              asm volatile(
                  "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                      smem_u32(&empty[s]))
                  : "memory");
            }
          }
          // this half's accumulator is ready (or the pipeline was abandoned)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(&acc_full[h]))
              : "memory");
        }
      }
    }
  } else {
    // epilogue warp: TMEM lanes 32 q .. 32 q + 31, column chunks ch = cg, cg + 4, ...
    const int q = warp & 3, cg = warp >> 2;
    const int nch = (NB + 31) / 32;
    int64_t i = 0;
    bool dead = false;
    for (int64_t w = blockIdx.x; w < npairs; w += gridDim.x, ++i) {
      // the previous pair's phase 3 (reads of S) is complete in every warp
      epi_bar();
      if (!dead && *abort_flag) dead = true;
      __nv_bfloat16* op = gp + w * out_ld;
      __nv_bfloat16* om = gm + w * out_ld;
      for (int h = 0; h < H; ++h) {
        if (!dead) {
          const bool ok = mbar_wait(smem_u32(&acc_full[h]), (uint32_t)(i & 1), err, 14);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (!ok || *abort_flag) {
            *abort_flag = 1;
            dead = true;
          }
        }
        const int cw = h * BM + q * 32;  // first row of this warp
        const int c = cw + lane;
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * BN);
        // phase 1: upper triangle W[c][d], d > c, to shared memory
        if (!dead && cw < v) {
          // S index of (c, d) is base_c + d
          const int base_c = c * (v - 1) - c * (c - 1) / 2;
          for (int ch = cg; ch < nch; ch += 4) {
            if (ch * 32 + 31 <= cw) continue;  // warp-uniform: no d > c here
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(ch * 32), r);
            if (c < v) {
              if (HS) {
                __nv_bfloat16* Sr = Sh + base_c + ch * 32;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                  const int d = ch * 32 + j;
                  if (d > c && d < v) Sr[j] = __float2bfloat16(__uint_as_float(r[j]));
                }
              } else {
                float* Sr = S + base_c + ch * 32;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                  const int d = ch * 32 + j;
                  if (d > c && d < v) Sr[j] = __uint_as_float(r[j]);
                }
              }
            }
          }
        }
        epi_bar();
        // phase 2: lower triangle d <= c with the stored transpose, packed in place
        if (!dead && cw < v) {
          for (int ch = cg; ch < nch; ch += 4) {
            if (ch * 32 > cw + 31) continue;  // warp-uniform: every d > every c
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(ch * 32), r);
            // S index of (d, c) is base_d + c; base_d is the same in every lane
            int base_d = (ch * 32) * (v - 1) - (ch * 32) * (ch * 32 - 1) / 2;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int d = ch * 32 + j;
              if (d <= c && c < v) {
                const float x = __uint_as_float(r[j]);
                const int qi = base_d + c;
                float sp, sm;
                if (d == c) {
                  sp = 2.0f * x;
                  sm = 0.0f;
                } else {
                  // W[d][c]
                  const float u = HS ? __bfloat162float(Sh[qi]) : S[qi];
                  sp = u + x;
                  sm = u - x;
                }
                const __nv_bfloat16 hp = __float2bfloat16(sp), hm = __float2bfloat16(sm);
                if (HS) {
                  Sh[qi] = hp;
                  om[qi] = hm;   // consecutive lanes: consecutive qi
                } else {
                  Su[qi] = (uint32_t)__bfloat16_as_ushort(hp) |
                           ((uint32_t)__bfloat16_as_ushort(hm) << 16);
                  if (nsl > 1) {
                    op[out_sstride + qi] = __float2bfloat16(sp - __bfloat162float(hp));
                    om[out_sstride + qi] = __float2bfloat16(sm - __bfloat162float(hm));
                  }
                }
              }
              base_d += v - 1 - d;
            }
          }
        }
        // this half's accumulator is read: hand it back to the MMA issuer
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0 && !dead)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[h]))
                       : "memory");
      }
      // phase 3: the packed triangle to the pair's two rows
      epi_bar();
      if (!dead) {
        const uint4* S4 = (const uint4*)Su;
        if (HS) {
          // eight G+ values per 16-byte load and store
          for (int64_t g8 = threadIdx.x; g8 < P8; g8 += LB_EPI * 32)
            *(uint4*)(op + 8 * g8) = S4[g8];
        } else {
          for (int64_t g4 = threadIdx.x; g4 < P4; g4 += LB_EPI * 32) {
            const uint4 e = S4[g4];
            uint2 pp, mm;
            pp.x = (e.x & 0xffffu) | (e.y << 16);
            pp.y = (e.z & 0xffffu) | (e.w << 16);
            mm.x = (e.x >> 16) | (e.y & 0xffff0000u);
            mm.y = (e.z >> 16) | (e.w & 0xffff0000u);
            *(uint2*)(op + 4 * g4) = pp;
            *(uint2*)(om + 4 * g4) = mm;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
      throw CudaError("cuTensorMapEncodeTiled entry point unavailable");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

CUtensorMap make_map(const void* base, int64_t rows_pad, int64_t k_pad, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)k_pad, (cuuint64_t)rows_pad};
  cuuint64_t strides[1] = {(cuuint64_t)(k_pad * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaError("cuTensorMapEncodeTiled failed: " + std::to_string(r));
  return m;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// row-major BF16 [rows][ld] with the contraction index K (extent k_ext) fastest
CUtensorMap make_map_ld(const void* base, int64_t rows, int64_t k_ext, int64_t ld, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)k_ext, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaError("cuTensorMapEncodeTiled failed: " + std::to_string(r));
  return m;
}

template <int MODE>
void set_mlp_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<4, 4, MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_bytes(4, 4));
  if (e != cudaSuccess) throw CudaError(std::string("tc smem attribute: ") + cudaGetErrorString(e));
}

}  // namespace

TcGemm::TcGemm(cudaStream_t st, int precision) : st_(st) {
  nslices_ = precision == 1 ? 2 : 1;
  if (cudaMalloc(&d_err_, sizeof(int)) != cudaSuccess) throw OomError("tc error flag");
  cudaMemsetAsync(d_err_, 0, sizeof(int), st_);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sm_count_, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sm_count_ < 1)
    throw CudaError("tc: cannot query the multiprocessor count");
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<4, 4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_bytes(4, 4));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_gemm<3, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes(3, 8));
  if (e != cudaSuccess) throw CudaError(std::string("tc smem attribute: ") + cudaGetErrorString(e));
  set_mlp_smem<MLP_HIDDEN>();
  set_mlp_smem<MLP_OUTPUT>();
  set_mlp_smem<MLP_RELU_BACK>();
  set_mlp_smem<MLP_PARTIAL>();
}

int TcGemm::mlp_gemm(int mode, const void* A, int64_t a_rows, int64_t lda, const void* B,
                     int64_t b_rows, int64_t ldb, int64_t M, int64_t N, int64_t K, int splits,
                     const MlpEpi& e) {
  if (M < 1 || N < 1 || K < 1 || a_rows < round_up(M, BM) || b_rows < round_up(N, BN) ||
      lda % 8 || ldb % 8 || lda < std::max<int64_t>(K, BK) || ldb < std::max<int64_t>(K, BK))
    throw std::runtime_error("mlp_gemm: bad operand shape");
  if (mode != MLP_PARTIAL) splits = 1;
  // K >= 64: the map's extent is K and TMA reads zeros past it; K < 64: the
  // caller has zeroed columns K .. 63
  const int64_t k_ext = std::max<int64_t>(K, BK);
  CUtensorMap ma = make_map_ld(A, a_rows, k_ext, lda, BM);
  CUtensorMap mb = make_map_ld(B, b_rows, k_ext, ldb, BN);
  const int64_t mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
  const int nk = (int)((k_ext + BK - 1) / BK);
  splits = std::max(1, std::min(splits, nk));
  const int kbs = (nk + splits - 1) / splits;
  splits = (nk + kbs - 1) / kbs;
  const int64_t items = mt * nt * splits;
  const int grid = (int)std::min<int64_t>(items, sm_count_);
  const int64_t split_stride = M * e.ldf;
  const size_t sm = smem_bytes(4, 4);
  switch (mode) {
    case MLP_HIDDEN:
      k_tc_gemm<4, 4, MLP_HIDDEN><<<grid, 192, sm, st_>>>(ma, mb, M, N, mt, nt, 0, items, nk, kbs,
                                                          1.0, nullptr, split_stride, OutView(),
                                                          0, d_err_, e);
      break;
    case MLP_OUTPUT:
      k_tc_gemm<4, 4, MLP_OUTPUT><<<grid, 192, sm, st_>>>(ma, mb, M, N, mt, nt, 0, items, nk, kbs,
                                                          1.0, nullptr, split_stride, OutView(),
                                                          0, d_err_, e);
      break;
    case MLP_RELU_BACK:
      k_tc_gemm<4, 4, MLP_RELU_BACK><<<grid, 192, sm, st_>>>(ma, mb, M, N, mt, nt, 0, items, nk,
                                                             kbs, 1.0, nullptr, split_stride,
                                                             OutView(), 0, d_err_, e);
      break;
    case MLP_PARTIAL:
      k_tc_gemm<4, 4, MLP_PARTIAL><<<grid, 192, sm, st_>>>(ma, mb, M, N, mt, nt, 0, items, nk,
                                                           kbs, 1.0, nullptr, split_stride,
                                                           OutView(), 0, d_err_, e);
      break;
    default:
      throw std::runtime_error("mlp_gemm: unknown epilogue");
  }
  count_launch();
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) throw CudaError(std::string("mlp_gemm launch: ") + cudaGetErrorString(err));
  return splits;
}

TcGemm::~TcGemm() {
  release(a_tmp_);
  release(b_tmp_);
  if (part_) cudaFree(part_);
  if (tune_buf_) cudaFree(tune_buf_);
  if (d_err_) cudaFree(d_err_);
}

void TcGemm::release(TcOperand& op) {
  if (op.data) cudaFree(op.data);
  op = TcOperand();
}

bool TcGemm::worthwhile(int64_t nb, int64_t M, int64_t N, int64_t K) const {
  // FP64 FMAs run at about 1/1000 of the BF16 tensor rate here, so even small
  // or skinny contractions (padded to 128 x 256 x 64 tiles, e.g. N = 6 trial
  // vectors) are cheaper as a conversion plus one tensor-core launch;
  // matrix-vector shapes stay on the memory-bound FP64 kernels
  return nb == 1 && M >= 2 && N >= 2 && (double)M * N * K >= 1.0e6;
}

void TcGemm::convert(const MatView& X, int64_t rows, int64_t K, TcOperand& out, int64_t spare) {
  const int64_t rp = round_up(rows + spare, BN), kp = round_up(K, BK);
  const size_t need = (size_t)rp * kp * 2 * nslices_;
  if (out.bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st_, &cs);
    if (cs != cudaStreamCaptureStatusNone)
      throw std::runtime_error("tensor-core buffer growth during graph capture (warm-up missing)");
    if (out.data) {
      cudaStreamSynchronize(st_);
      cudaFree(out.data);
      out.data = nullptr;
    }
    if (cudaMalloc(&out.data, need) != cudaSuccess) {
      cudaGetLastError();
      throw OomError("tensor-core operand buffer of " + std::to_string(need) + " bytes");
    }
    out.bytes = need;
  }
  out.rows = rows;
  out.k = K;
  out.rows_pad = rp;
  out.k_pad = kp;
  out.slices = nslices_;
  const int64_t tiles = (rp / CR) * (kp / CK);
  int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sm_count_ * 6));
  k_split_bf16_view<<<grid, 256, 0, st_>>>(X, rows, K, rp, kp, nslices_, (__nv_bfloat16*)out.data);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string("split_bf16: ") + cudaGetErrorString(e));
}

void TcGemm::prepare_operand(const double* X, int64_t rows, int64_t K, TcOperand& out) {
  convert(MatView::dense(X, rows, K), rows, K, out);
}

void TcGemm::prepare_operand_view(const MatView& X, int64_t rows, int64_t K, TcOperand& out) {
  convert(X, rows, K, out);
}

void TcGemm::check_error() {
  int h = 0;
  cudaMemcpyAsync(&h, d_err_, sizeof(int), cudaMemcpyDeviceToHost, st_);
  cudaStreamSynchronize(st_);
  if (h != 0) {
    cudaMemsetAsync(d_err_, 0, sizeof(int), st_);
    throw CudaError("tensor-core pipeline wait expired (code " + std::to_string(h) + ")");
  }
}

void TcGemm::run(const TcOperand& A, int sa, const TcOperand& B, int sb, int64_t M, int64_t N,
                 double alpha, double* C, int64_t split_stride, const OutView& ov,
                 bool accumulate, int splits, int kbs, int variant, int nfast) {
  if (A.k_pad != B.k_pad) throw std::runtime_error("tc: K mismatch");
  const __nv_bfloat16* a = (const __nv_bfloat16*)A.data + (size_t)sa * A.rows_pad * A.k_pad;
  const __nv_bfloat16* b = (const __nv_bfloat16*)B.data + (size_t)sb * B.rows_pad * B.k_pad;
  CUtensorMap ma = make_map(a, A.rows_pad, A.k_pad, BM);
  CUtensorMap mb = make_map(b, B.rows_pad, B.k_pad, BN);
  const int64_t mt = (M + BM - 1) / BM, nt = B.rows_pad / BN;
  const int64_t items = mt * nt * splits;
  const int grid = (int)std::min<int64_t>(items, sm_count_);
  const int nk = (int)(A.k_pad / BK);

  if (variant == 1)
    k_tc_gemm<3, 8><<<grid, 320, smem_bytes(3, 8), st_>>>(ma, mb, M, N, mt, nt, nfast, items, nk,
                                                          kbs, alpha, C, split_stride, ov,
                                                          accumulate ? 1 : 0, d_err_, MlpEpi());
  else
    k_tc_gemm<4, 4><<<grid, 192, smem_bytes(4, 4), st_>>>(ma, mb, M, N, mt, nt, nfast, items, nk,
                                                          kbs, alpha, C, split_stride, ov,
                                                          accumulate ? 1 : 0, d_err_, MlpEpi());
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string("tc_gemm launch: ") + cudaGetErrorString(e));
}

// slice pairs (i, j) with i + j < slices, largest first
static void slice_pairs(int s, std::vector<std::pair<int, int>>& out) {
  out.clear();
  for (int tot = 0; tot < s; ++tot)
    for (int i = 0; i <= tot; ++i) out.push_back({i, tot - i});
}

void TcGemm::gemm_prepared_b(int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                             const TcOperand& B, double* C, bool check) {
  convert(MatView::dense(A, M, K), M, K, a_tmp_);
  gemm_ops(M, N, alpha, a_tmp_, B, C, OutView::dense(N), false);
  (void)check;  // the error flag is read by the backend at each synchronisation
}

namespace {

// FNV-1a over the levels and strides of an output view
uint64_t view_hash(const OutView& ov) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](int64_t x) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((x >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  mix(ov.nr);
  mix(ov.nc);
  for (int l = 0; l < ov.nr; ++l) { mix(ov.re[l]); mix(ov.rs[l]); }
  for (int l = 0; l < ov.nc; ++l) { mix(ov.ce[l]); mix(ov.cs[l]); }
  return h;
}

// 1 + the largest offset an M x N result can reach through the view (an upper
// bound), or -1 for views with negative strides
int64_t view_span(const OutView& ov, int64_t M, int64_t N) {
  auto bound = [](int n, const int64_t* ext, const int64_t* str, int64_t count) -> int64_t {
    int64_t inner = 1, b = 0;
    for (int l = 1; l < n; ++l) {
      if (ext[l] < 1 || str[l] < 0) return -1;
      inner *= ext[l];
      b += (ext[l] - 1) * str[l];
    }
    if (str[0] < 0) return -1;
    return b + str[0] * ((count - 1) / inner);
  };
  const int64_t r = bound(ov.nr, ov.re, ov.rs, M), c = bound(ov.nc, ov.ce, ov.cs, N);
  if (r < 0 || c < 0) return -1;
  return r + c + 1;
}

}  // namespace

void TcGemm::gemm_ops(int64_t M, int64_t N, double alpha, const TcOperand& A, const TcOperand& B,
                      double* C, const OutView& ov, bool accumulate) {
  TcShape s;
  s.M = M;
  s.n_pad = B.rows_pad;
  s.nk = (int)(A.k_pad / BK);
  s.slices = nslices_;
  s.accumulate = accumulate ? 1 : 0;
  s.sm_count = sm_count_;
  s.view_hash = view_hash(ov);
  const int64_t mt = (M + BM - 1) / BM, nt = B.rows_pad / BN;
  const double abytes = (double)A.rows_pad * A.k_pad, bbytes = (double)B.rows_pad * B.k_pad;
  TcConfig cfg;
  if (!TcTuneTable::global().find(s, cfg)) {
    cfg = tc_default_config(s, mt, nt, abytes, bbytes);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st_, &cs);
    if (tune_ && cs == cudaStreamCaptureStatusNone) cfg = tune(s, M, N, alpha, A, B, ov, cfg);
  }
  execute(cfg, M, N, alpha, A, B, C, ov, accumulate);
}

void TcGemm::set_tune(bool on) {
  tune_ = on;
  if (!on && tune_buf_) {
    cudaStreamSynchronize(st_);
    cudaFree(tune_buf_);
    tune_buf_ = nullptr;
    tune_bytes_ = 0;
  }
}

TcConfig TcGemm::tune(const TcShape& s, int64_t M, int64_t N, double alpha, const TcOperand& A,
                      const TcOperand& B, const OutView& ov, const TcConfig& fallback) {
  const int64_t span = view_span(ov, M, N);
  if (span < 1) return fallback;
  if (tune_bytes_ < (size_t)span * sizeof(double)) {
    cudaStreamSynchronize(st_);
    if (tune_buf_) cudaFree(tune_buf_);
    tune_buf_ = nullptr;
    tune_bytes_ = 0;
    if (cudaMalloc(&tune_buf_, (size_t)span * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fallback;
    }
    tune_bytes_ = (size_t)span * sizeof(double);
  }
  const int64_t mt = (M + BM - 1) / BM, nt = B.rows_pad / BN;
  const double abytes = (double)A.rows_pad * A.k_pad, bbytes = (double)B.rows_pad * B.k_pad;
  struct Events {   // destroyed on every exit, including a CUDA error thrown below
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) {
    cudaGetLastError();
    return fallback;
  }
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  TcConfig best = fallback;
  double best_us = 1e300;
  const int reps = 3;
  // candidates write the real view into a scratch buffer of its span (with the
  // real accumulate mode), so the caller's output is untouched
  for (const TcConfig& c : tc_candidates(s, mt, nt, abytes, bbytes)) {
    try {
      execute(c, M, N, alpha, A, B, tune_buf_, ov, s.accumulate != 0);
      cudaEventRecord(e0, st_);
      for (int r = 0; r < reps; ++r) execute(c, M, N, alpha, A, B, tune_buf_, ov, s.accumulate != 0);
      cudaEventRecord(e1, st_);
      cudaEventSynchronize(e1);
    } catch (const OomError&) {
      continue;
    }
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const double us = 1e3 * ms / reps;
    if (us < best_us) {
      best_us = us;
      best = c;
    }
  }
  check_error();
  TcTuneTable::global().put(s, best, best_us);
  return best;
}

void TcGemm::execute(const TcConfig& cfg, int64_t M, int64_t N, double alpha, const TcOperand& A,
                     const TcOperand& B, double* C, const OutView& ov, bool accumulate) {
  std::vector<std::pair<int, int>> pairs;
  slice_pairs(nslices_, pairs);
  const int nk = (int)(A.k_pad / BK);
  const int splits = cfg.splits, kbs = cfg.kbs;
  // accumulate the small slice products first, the leading one last
  if (splits == 1) {
    for (size_t p = pairs.size(); p-- > 0;)
      run(A, pairs[p].first, B, pairs[p].second, M, N, alpha, C, 0, ov,
          accumulate || p + 1 != pairs.size(), 1, nk, cfg.variant, cfg.nfast);
    return;
  }
  const size_t need = (size_t)splits * M * N * sizeof(double);
  if (part_bytes_ < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st_, &cs);
    if (cs != cudaStreamCaptureStatusNone)
      throw std::runtime_error("tensor-core buffer growth during graph capture (warm-up missing)");
    if (part_) {
      cudaStreamSynchronize(st_);
      cudaFree(part_);
      part_ = nullptr;
      part_bytes_ = 0;
    }
    if (cudaMalloc(&part_, need) != cudaSuccess) {
      cudaGetLastError();
      throw OomError("split-K buffer of " + std::to_string(need) + " bytes");
    }
    part_bytes_ = need;
  }
  for (size_t p = pairs.size(); p-- > 0;)
    run(A, pairs[p].first, B, pairs[p].second, M, N, alpha, part_, M * N, OutView::dense(N),
        p + 1 != pairs.size(), splits, kbs, cfg.variant, cfg.nfast);
  const int64_t n = M * N;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count_ * 16));
  k_sum_splits<<<grid, 256, 0, st_>>>(M, N, splits, part_, C, ov, accumulate ? 1 : 0);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string("sum_splits: ") + cudaGetErrorString(e));
}

void TcGemm::alloc_operand(int64_t rows, int64_t k, int slices, TcOperand& out) {
  const int64_t rp = round_up(std::max<int64_t>(rows, 1), BN), kp = round_up(std::max<int64_t>(k, 1), BK);
  const size_t need = (size_t)rp * kp * 2 * slices;
  if (out.bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st_, &cs);
    if (cs != cudaStreamCaptureStatusNone)
      throw std::runtime_error("tensor-core buffer growth during graph capture (warm-up missing)");
    if (out.data) {
      cudaStreamSynchronize(st_);
      cudaFree(out.data);
      out.data = nullptr;
      out.bytes = 0;
    }
    if (cudaMalloc(&out.data, need) != cudaSuccess) {
      cudaGetLastError();
      throw OomError("tensor-core operand buffer of " + std::to_string(need) + " bytes");
    }
    out.bytes = need;
    // the K padding must read as zeros; the kernels never write it
    if (cudaMemsetAsync(out.data, 0, need, st_) != cudaSuccess)
      throw CudaError("tensor-core operand memset failed");
  } else if (out.rows_pad != rp || out.k_pad != kp || out.slices != slices) {
    if (cudaMemsetAsync(out.data, 0, need, st_) != cudaSuccess)
      throw CudaError("tensor-core operand memset failed");
  }
  out.rows = rows;
  out.k = k;
  out.rows_pad = rp;
  out.k_pad = kp;
  out.slices = slices;
}

void TcGemm::prepare_ladder_lt(const double* L, int o, int v, int J, TcOperand& out) {
  const int64_t n = (int64_t)o + v;
  MatView X;  // element (r = p v + q, k = J) = L[J][o + p][o + q]
  X.p = L + o * n + o;
  X.n2r = v;
  X.sr1 = n;
  X.sr2 = 1;
  X.sk2 = n * n;
  convert(X, (int64_t)v * v, J, out, 256);
  // the spare rows only feed accumulator rows and columns that are never
  // read; zero them so that they hold no stale bits either
  const int64_t used = (int64_t)v * v;
  for (int s = 0; s < out.slices; ++s) {
    char* base = (char*)out.data + ((size_t)s * out.rows_pad + used) * out.k_pad * 2;
    const size_t len = (size_t)(out.rows_pad - used) * out.k_pad * 2;
    if (cudaMemsetAsync(base, 0, len, st_) != cudaSuccess)
      throw CudaError("ladder operand memset failed");
  }
}

namespace {
int ladder_nb(int v) { return (int)round_up(v, 16); }
int ladder_stage_bytes(int v) { return A_BYTES + ladder_nb(v) * BK * 2; }
// the upper triangle in shared memory: FP32 entries (two slices) or BF16 (one)
int ladder_tri_bytes(int v, int nsl) {
  return nsl == 1 ? (int)round_up((int64_t)v * (v + 1) / 2, 8) * 2
                  : (int)round_up((int64_t)v * (v + 1) / 2, 4) * 4;
}
constexpr int kSmemMax = 232448;  // dynamic shared memory a block may opt in to
int ladder_stages(int v, int nsl) {
  const int room = kSmemMax - 1024 - 256 - ladder_tri_bytes(v, nsl);
  return std::min(6, room / ladder_stage_bytes(v));
}
}  // namespace

int TcGemm::ladder_build_max_v() {
  // the two-slice form has the larger triangle: every v up to this fits both
  int v = 2 * BM;
  while (v > 1 && ladder_stages(v, 2) < 2) --v;
  return v;
}

void TcGemm::ladder_build(const TcOperand& Lt, int v, const int* pairs, int64_t p_begin,
                          int64_t npairs, TcOperand& Gp, TcOperand& Gm) {
  if (npairs <= 0) return;
  if (v < 1 || v > ladder_build_max_v()) throw std::runtime_error("ladder build: v out of range");
  const int NB = ladder_nb(v), two = v > BM ? 1 : 0;
  const int stages = ladder_stages(v, Lt.slices);
  const int64_t Pv = (int64_t)v * (v + 1) / 2;
  if (Lt.rows != (int64_t)v * v || Lt.rows_pad < Lt.rows + 256)
    throw std::runtime_error("ladder build: Lt operand without its spare rows");
  if (Gp.k != Pv || Gm.k != Pv || Gp.rows < npairs || Gm.rows < npairs ||
      Gp.slices != Lt.slices || Gm.slices != Lt.slices || Gp.k_pad != Gm.k_pad ||
      Gp.rows_pad != Gm.rows_pad)
    throw std::runtime_error("ladder build: output operands of the wrong shape");
  // one map over all slices of Lt (slice s starts at row s * rows_pad); box
  // heights 128 (A: rows c) and NB (B: rows d)
  CUtensorMap ma = make_map(Lt.data, (int64_t)Lt.slices * Lt.rows_pad, Lt.k_pad, BM);
  CUtensorMap mb = make_map(Lt.data, (int64_t)Lt.slices * Lt.rows_pad, Lt.k_pad, NB);
  const int smem = 1024 + stages * ladder_stage_bytes(v) + 256 + ladder_tri_bytes(v, Lt.slices);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_ladder_build<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_ladder_build<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kSmemMax);
    if (e != cudaSuccess) throw CudaError(std::string("ladder build smem attribute: ") + cudaGetErrorString(e));
    attr_set = true;
  }
  const int nprod = Lt.slices == 1 ? 1 : 3;
  const int grid = (int)std::min<int64_t>(npairs, sm_count_);
  if (Lt.slices == 1)
    k_ladder_build<true><<<grid, LB_THREADS, smem, st_>>>(
        ma, mb, v, NB, two, (int)(Lt.k_pad / BK), nprod, Lt.rows_pad, stages, pairs, p_begin,
        npairs, (__nv_bfloat16*)Gp.data, (__nv_bfloat16*)Gm.data, Gp.k_pad,
        Gp.rows_pad * Gp.k_pad, Lt.slices, d_err_);
  else
    k_ladder_build<false><<<grid, LB_THREADS, smem, st_>>>(
        ma, mb, v, NB, two, (int)(Lt.k_pad / BK), nprod, Lt.rows_pad, stages, pairs, p_begin,
        npairs, (__nv_bfloat16*)Gp.data, (__nv_bfloat16*)Gm.data, Gp.k_pad,
        Gp.rows_pad * Gp.k_pad, Lt.slices, d_err_);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string("ladder build launch: ") + cudaGetErrorString(e));
}

void TcGemm::gemm(int64_t nb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                  const double* B, double* C) {
  if (nb != 1) throw std::runtime_error("tc: batched GEMM not supported");
  convert(MatView::dense(B, N, K), N, K, b_tmp_);
  gemm_prepared_b(M, N, K, alpha, A, b_tmp_, C);
}

}  // namespace sccsd
