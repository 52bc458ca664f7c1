// panel.cu -- the level-1 product Y = A X for many right-hand sides on the tensor cores.
//
// Sec. 3.1 writes the H2 product as small dense products: the near blocks D_ts x_s, the
// couplings S_ts x_hat_s, and the transfers x_hat_l = U_l^T x_l, x_hat_p += E_c^T x_hat_c
// (upward), y_hat_c = y_row_c + E_c y_hat_p and y_l = y_near_l + U_l y_hat_l (downward).
// With W right-hand sides each of them contracts a 64 x 64 block with a 64 x W panel,
// which is tensor-core work. Every step here is one launch of k_panel_mma:
//
//   D_row [W x 64] = C_row + sum over entries e of row:  X_col(e)^T [W x 64] * B_e [64 x 64]
//
// with one CTA per output row, D in tensor memory (TMEM, 128 lanes = the W columns of
// the panel, 64 FP32 columns), and W = 128 so that every tcgen05.mma is the full
// 128 x 64 x 8 shape. Operands sit in shared memory in the 128-byte-swizzled K-major
// layout of tcgen05 shared-memory descriptors. Panels that later steps read as operands
// are written once, by their producer, already split into their TF32 head and tail tiles
// in that layout (64 KB per panel), so that one thread moves an entry's panel into shared
// memory with bulk copies (cp.async.bulk, completion on an mbarrier); the blocks are read
// through registers, where the CTA's threads rearrange and split them.
//
// Precision: the blocks are the FP32 copy. Each FP32 operand a is split into
// a_hi = tf32(a) (rounded to nearest) and a_lo = tf32(a - a_hi), and every block product
// is the sum of three TF32 products a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped
// a_lo b_lo is below 2^-22 |a b|). The tensor core's own FP32 accumulation does not round
// to nearest, and its error grows with the number of MMAs summed into one accumulator:
// summed over a whole block row (hundreds of MMAs) it left errors near 1e-5. So each
// entry's products go to fresh TMEM accumulators (the head products in one, the two
// correction products in another, 8 and 16 MMAs), which the threads read after the
// entry and add, rounding to nearest, into registers: FP32-level accuracy. Two sets of
// accumulators alternate between entries, so that entry j - 1's are read while entry j's
// MMAs run.
//
// The symmetric operators are stored as their upper triangle. Here they are read in full:
// block (t, s), s > t, is staged for row t (read by rows) and again, transposed, for row s
// (read by columns), so that every output row is written once, without atomics, at the
// price of reading each off-diagonal block twice.
#include <algorithm>

#include "internal.h"

namespace h2mg {

namespace {

constexpr int PW = 128;                          // right-hand sides per panel (MMA M)
constexpr int PK = 64;                           // block edge (MMA N and contraction length)
constexpr uint32_t kTileA = PW * PK * 4;         // one A tile (hi or lo): 32 KB
constexpr uint32_t kTileB = PK * PK * 4;         // one B tile: 16 KB
constexpr uint32_t kStage = 2 * kTileA + 2 * kTileB;
constexpr uint32_t kPanelSP = 2 * kTileA;        // a split panel: head tile, then tail tile
constexpr uint32_t kDynSmem = kStage + 1024;     // + alignment of the swizzle atoms
constexpr uint32_t kTmemCols = 256;              // 2 sets x 2 FP32 accumulators of 64 columns x 128 lanes
// Instruction descriptor of tcgen05.mma kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(PK >> 3) << 17) |
                            ((uint32_t)(PW >> 4) << 24);
constexpr long long kWaitCycles = 1ll << 32;     // bound of every wait (about two seconds)

enum : unsigned char { BM_NAT = 0, BM_ROW = 1, BM_COL = 2 };

struct PanelArgs {
  const int* rowptr;                 // [nrows + 1]
  const int* col;                    // [nnz] input panel of the entry
  const float* const* blk;           // [nnz] 64 x 64 FP32 block of the entry
  const unsigned char* mode;         // [nnz] BM_*: how the block is read
  const char* xin;                   // input panels, split (kPanelSP bytes each)
  const float* cin;                  // addend panels, plain FP32 [W][64] (row + cin_off), or null
  void* out;                         // output panels (row + out_off), or null: scatter
  int out_split;                     // 1: outputs split like the inputs, 0: plain FP32
  int64_t cin_off, out_off;
  const int* leafoff;                // scatter: leaf offsets in tree order
  const int* perm;                   //          tree position -> user index
  double* y;                         //          float64 columns, leading dimension ldy
  int64_t ldy;
  int nr;                            //          columns of the panel in use
  int* flag;                         // set to 1 when a wait ran out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in a K-major tile of R rows x 64 FP32 with the 128-byte
// swizzle: two 32-element K halves of R x 128 B each; inside a half, 8-row groups of
// 1024 B, rows 128 B apart, and the 16-byte chunk c of row r stored at chunk c ^ (r & 7).
template <int R>
__device__ __forceinline__ uint32_t swz(int row, int k) {
  return (uint32_t)((k >> 5) * (R * 128) + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((k & 31) >> 2) ^ (row & 7)) << 4) + ((k & 3) << 2));
}

// Shared-memory matrix descriptor of tcgen05 for that layout: start address >> 4
// (bits 0-13), leading byte offset (unused by swizzled K-major operands; 16 B) at bit 16,
// stride byte offset between 8-row groups (1024 B) at bit 32, the fixed value 1 at bit
// 46, swizzle mode 2 (128 B) at bit 61.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Round an FP32 value to TF32 (10 fraction bits), to nearest with ties away from zero:
// add half a unit of the 13 dropped bits to the magnitude's bit pattern (a carry moves
// into the exponent correctly) and clear them. Two integer operations, where a
// conversion instruction runs on the slower conversion pipe.
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void split4(const float4& v, float4& hi, float4& lo) {
  hi.x = tf32_rn(v.x);
  hi.y = tf32_rn(v.y);
  hi.z = tf32_rn(v.z);
  hi.w = tf32_rn(v.w);
  lo.x = tf32_rn(v.x - hi.x);
  lo.y = tf32_rn(v.y - hi.y);
  lo.z = tf32_rn(v.z - hi.z);
  lo.w = tf32_rn(v.w - hi.w);
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Global -> shared bulk copy (16-byte aligned, a multiple of 16 bytes) whose completion
// counts `bytes` on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
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

// Waits for the phase of the given parity to complete; 0 after kWaitCycles without it.
__device__ __forceinline__ int mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWaitCycles) return 0;
  return 1;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d), "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// acc += the entry's head and correction accumulators (columns c0..c0+31 of this
// thread's lane), their sum rounded to nearest.
__device__ __forceinline__ void tmem_accumulate(uint32_t taddr, float* acc) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    uint32_t h[16], c[16];
    tmem_ld16(taddr + 16 * q, h);
    tmem_ld16(taddr + 64 + 16 * q, c);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[16 * q + j] += __uint_as_float(h[j]) + __uint_as_float(c[j]);
  }
}

__device__ __forceinline__ float pick(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Float4 of the swizzled 64 x 64 FP32 block layout (one float4 = rows r0..r0+3 of one
// column c; position (cc << 3) | g holds column c0 + cc and rows 8 g + ..) that thread
// lane `lane` of a warp loads for the row / column reads: a permutation inside the warp's
// 512-byte segment. The four lanes holding the same rows are neighbours (lane & ~3, the
// 4 x 4 transposition below). Each group of 8 lanes (one 16-byte store wavefront) takes
// the row groups g and g + 2 (g in 0, 1, 4, 5): their 16-byte chunks differ in the third
// bit of the swizzle phase, so the column reads store without bank conflicts (the row
// reads with two lanes per bank).
__device__ __forceinline__ int swz_lane_pos(int lane) {
  const int cc = lane & 3, m = lane >> 3, b = (lane >> 2) & 1;
  const int g = (m & 1) + 4 * (m >> 1) + 2 * b;
  return (cc << 3) | g;
}

// Row (r0 + cc) of the 4 x 4 tile whose columns c0..c0+3 the four lanes (lane & ~3) + j
// hold as float4s of rows r0..r0+3 (lane (lane & ~3) + cc holds column c0 + cc).
__device__ __forceinline__ float4 transpose4(const float4& v, int lane) {
  const int cc = lane & 3;
  float r[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int src = (cc + k) & 3;              // lane read in this round
    const float send = pick(v, (cc - k) & 3);  // the element the reader (cc - k) wants from us
    r[k] = __shfl_sync(0xffffffffu, send, (lane & ~3) | src);
  }
  // r[k] is column c0 + ((cc + k) & 3) of our row
  float o[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int k = (m - cc) & 3;
    o[m] = k == 0 ? r[0] : (k == 1 ? r[1] : (k == 2 ? r[2] : r[3]));
  }
  return make_float4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Global loads of one entry's block (4 float4 per thread, position by mode).
__device__ __forceinline__ void load_block(const PanelArgs& a, int e, int tid, float4* pb) {
  const float4* B = reinterpret_cast<const float4*>(a.blk[e]);
  const int q0 = a.mode[e] == BM_NAT ? tid : ((tid & ~31) | swz_lane_pos(tid & 31));
#pragma unroll
  for (int i = 0; i < 4; ++i) pb[i] = __ldg(B + q0 + 256 * i);
}

// One thread: the entry's split panel (head and tail tiles, 64 KB) into the A tiles.
__device__ __forceinline__ void copy_panel(const PanelArgs& a, int e, uint32_t sA, uint32_t bar) {
  const char* src = a.xin + (size_t)a.col[e] * kPanelSP;
  mbar_expect_tx(bar, kPanelSP);
#pragma unroll
  for (int c = 0; c < 4; ++c) bulk_g2s(sA + c * (kPanelSP / 4), src + c * (kPanelSP / 4), kPanelSP / 4, bar);
}

// Shared-memory stores of one entry's block as the B operand in "n-rows" form (row n
// holds the 64 contraction elements of output column n), as TF32 head and tail tiles.
__device__ __forceinline__ void store_block(uint8_t* sm, int md, int tid, const float4* pb) {
  uint8_t* Bh = sm + 2 * kTileA;
  uint8_t* Bl = Bh + kTileB;
  float4 hi, lo;
  const int lane = tid & 31;
  if (md == BM_NAT) {
    // natural column-major block whose column n is row n of the operand: float4
    // q = tid + 256 i is row (tid >> 4) + 16 i, elements 4 (tid & 15) .., so the rows
    // advance by two 8-row groups (2048 B) per i and the swizzle phase stays
    const uint32_t offb = swz<PK>(tid >> 4, (tid & 15) << 2);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      split4(pb[i], hi, lo);
      *reinterpret_cast<float4*>(Bh + offb + 2048 * i) = hi;
      *reinterpret_cast<float4*>(Bl + offb + 2048 * i) = lo;
    }
    return;
  }
  // swizzled block: float4 index q holds rows r0..r0+3 of column c; with
  // q = (warp base | lane position) + 256 i the column advances by 16 per i
  const int q0 = (tid & ~31) | swz_lane_pos(lane);
  const int l = q0 & 31, tk = q0 >> 5;
  const int c0 = 4 * (tk >> 1) + (l >> 3), r0 = 8 * (l & 7) + 4 * (tk & 1);
  if (md == BM_COL) {
    const uint32_t offb = swz<PK>(c0, r0);          // column c of the block is operand row c
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      split4(pb[i], hi, lo);
      *reinterpret_cast<float4*>(Bh + offb + 2048 * i) = hi;
      *reinterpret_cast<float4*>(Bl + offb + 2048 * i) = lo;
    }
  } else {
    const int cc = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 v = transpose4(pb[i], lane);   // row r0 + cc, columns c - cc .. c - cc + 3
      const uint32_t off = swz<PK>(r0 + cc, c0 + 16 * i - cc);
      split4(v, hi, lo);
      *reinterpret_cast<float4*>(Bh + off) = hi;
      *reinterpret_cast<float4*>(Bl + off) = lo;
    }
  }
}

__global__ void __launch_bounds__(256, 2) k_panel_mma(PanelArgs a) {
  extern __shared__ uint8_t dsm[];
  __shared__ uint64_t bar;      // the entry's MMAs have completed
  __shared__ uint64_t bar_a;    // the entry's panel has arrived
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = blockIdx.x;
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  uint8_t* sm = dsm + (base - smem_u32(dsm));
  const uint32_t sAh = base, sAl = base + kTileA, sBh = base + 2 * kTileA, sBl = sBh + kTileB;
  const int e0 = a.rowptr[row], ne = a.rowptr[row + 1] - e0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(&bar));
    mbar_init(smem_u32(&bar_a));
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;

  // this thread's share of D: lane w = 32 (warp % 4) + lane, columns 32 (warp / 4) ..
  const int qd = warp & 3, h = warp >> 2;
  const int w = 32 * qd + lane;                       // right-hand side of this thread
  const uint32_t tacc = tmem + ((uint32_t)(32 * qd) << 16) + 32 * h;
  float v[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = 0.f;
  float4 pb[4];
  int issued = 0;         // entries whose MMAs were committed
  int copied = 0;         // thread 0: panels whose copy was started
  int t0ok = 1;           // thread 0: every wait so far completed
  bool bad = false;
  if (ne > 0) {
    load_block(a, e0, tid, pb);
    if (tid == 0) {
      copy_panel(a, e0, sAh, smem_u32(&bar_a));
      copied = 1;
    }
  }
  for (int j = 0; j < ne; ++j) {
    if (j > 0) {
      // entry j - 1's products are complete: they have read the staging tiles
      if (tid == 0) t0ok &= mbar_wait(smem_u32(&bar), (uint32_t)((j - 1) & 1));
      if (__syncthreads_or(tid == 0 && !t0ok)) {
        bad = true;
        break;
      }
      if (tid == 0) {
        copy_panel(a, e0 + j, sAh, smem_u32(&bar_a));
        copied = j + 1;
      }
    }
    store_block(sm, a.mode[e0 + j], tid, pb);
    fence_async_smem();
    tc_fence_before();    // the reads of the set that entry j's products will overwrite
    __syncthreads();
    if (j + 1 < ne) load_block(a, e0 + j + 1, tid, pb);      // in flight during the products
    if (tid == 32 && j + 2 < ne) {                            // and the entry after, into L2
      prefetch_l2(a.blk[e0 + j + 2], PK * PK * 4);
      prefetch_l2(a.xin + (size_t)a.col[e0 + j + 2] * kPanelSP, kPanelSP);
    }
    if (tid == 0) {
      t0ok &= mbar_wait(smem_u32(&bar_a), (uint32_t)(j & 1));   // the panel is in place
      tc_fence_after();
      const uint32_t set = tmem + (uint32_t)(j & 1) * 128;
      if (t0ok) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          const uint32_t ta = p == 2 ? sAl : sAh, tb = p == 1 ? sBl : sBh;
          const uint32_t td = p == 0 ? set : set + 64;     // head / correction accumulator
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const uint64_t da = sw128_desc(ta + (s >> 2) * (PW * 128) + (s & 3) * 32);
            const uint64_t db = sw128_desc(tb + (s >> 2) * (PK * 128) + (s & 3) * 32);
            mma_tf32(td, da, db, (p == 2 || s > 0) ? 1u : 0u);
          }
        }
      }
      mma_commit(smem_u32(&bar));
    }
    if (j > 0) {
      // entry j - 1's accumulators, while entry j's products run
      tc_fence_after();
      tmem_accumulate(tacc + (uint32_t)((j - 1) & 1) * 128, v);
    }
    issued = j + 1;
  }
  if (issued > 0 && !bad) {
    if (tid == 0) t0ok &= mbar_wait(smem_u32(&bar), (uint32_t)((issued - 1) & 1));
    if (__syncthreads_or(tid == 0 && !t0ok)) {
      bad = true;
    } else {
      tc_fence_after();
      tmem_accumulate(tacc + (uint32_t)((issued - 1) & 1) * 128, v);
    }
  }
  if (bad && tid == 0) {
    // a wait ran out: one more bounded wait for the copies and products in flight before
    // the shared memory and the accumulators are released
    if (copied > 0) mbar_wait(smem_u32(&bar_a), (uint32_t)((copied - 1) & 1));
    if (issued > 0) mbar_wait(smem_u32(&bar), (uint32_t)((issued - 1) & 1));
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) atomicExch(a.flag, 1);
  } else {
    if (a.cin) {
      const float4* C = reinterpret_cast<const float4*>(a.cin + ((size_t)(row + a.cin_off) * PW + w) * PK + 32 * h);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float4 c = __ldg(C + j);
        v[4 * j] += c.x;
        v[4 * j + 1] += c.y;
        v[4 * j + 2] += c.z;
        v[4 * j + 3] += c.w;
      }
    }
    if (a.out && a.out_split) {
      // split panel: elements 32 h + 4 j .. of row w in the head and tail tiles
      char* O = reinterpret_cast<char*>(a.out) + (size_t)(row + a.out_off) * kPanelSP;
      float4 hi, lo;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        split4(make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]), hi, lo);
        const uint32_t off = swz<PW>(w, 32 * h + 4 * j);
        *reinterpret_cast<float4*>(O + off) = hi;
        *reinterpret_cast<float4*>(O + kTileA + off) = lo;
      }
    } else if (a.out) {
      float4* O = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.out) +
                                            ((size_t)(row + a.out_off) * PW + w) * PK + 32 * h);
#pragma unroll
      for (int j = 0; j < 8; ++j) O[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    } else {
      // row = leaf: stage [W][65] in the (now idle) A tiles, then write the leaf's points
      // of the nr columns in use to user order
      float* st = reinterpret_cast<float*>(sm);
#pragma unroll
      for (int j = 0; j < 32; ++j) st[w * 65 + 32 * h + j] = v[j];
      __syncthreads();
      const int p0 = a.leafoff[row], nl = a.leafoff[row + 1] - p0;
      for (int idx = tid; idx < nl * a.nr; idx += 256) {
        const int i = idx % nl, ww = idx / nl;
        a.y[(int64_t)a.perm[p0 + i] + (int64_t)ww * a.ldy] = (double)st[ww * 65 + i];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Float64 columns (user order, leading dimension ldx) -> split point panels (one per
// leaf), zero in padded slots and unused columns.
__global__ void k_panel_in(const double* __restrict__ x, int64_t ldx, int nr, const int* __restrict__ leafoff,
                           const int* __restrict__ perm, int nleaf, char* __restrict__ xp) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t l = idx / (PW * PK);
  if (l >= nleaf) return;
  const int i = (int)(idx % PK), w = (int)((idx / PK) % PW);
  const int p0 = leafoff[l], nl = leafoff[l + 1] - p0;
  float v = 0.f;
  if (w < nr && i < nl) v = (float)x[(int64_t)perm[p0 + i] + (int64_t)w * ldx];
  const float hi = tf32_rn(v);
  char* P = xp + (size_t)l * kPanelSP + swz<PW>(w, i);
  *reinterpret_cast<float*>(P) = hi;
  *reinterpret_cast<float*>(P + kTileA) = tf32_rn(v - hi);
}

}  // namespace

// ----------------------------------------------------------------------------- host plan
struct PanelCSR {
  int nrows = 0;
  int64_t nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  const float** blk = nullptr;
  unsigned char* mode = nullptr;
};

struct PanelPlan {
  PanelCSR lup, near, coup, lfin;
  std::vector<PanelCSR> up, down;   // index: tree level ell
  char *xp = nullptr, *xc = nullptr, *yc = nullptr;   // split panels (operands of later steps)
  float *yr = nullptr, *yp = nullptr;                 // plain panels (addends)
};

void destroy_panel_plan(Matrix& M) {
  delete M.panel;
  M.panel = nullptr;
}

namespace {

struct HostList {
  std::vector<int> rowptr{0}, col;
  std::vector<const float*> blk;
  std::vector<unsigned char> mode;
  void add(int c, const float* b, unsigned char m) {
    col.push_back(c);
    blk.push_back(b);
    mode.push_back(m);
  }
  void end_row() { rowptr.push_back((int)col.size()); }
};

PanelCSR upload_list(Matrix& M, const HostList& H) {
  PanelCSR C;
  C.nrows = (int)H.rowptr.size() - 1;
  C.nnz = (int64_t)H.col.size();
  cudaStream_t s = M.stream;
  auto up = [&](const void* src, size_t bytes) {
    void* d = M.alloc(std::max<size_t>(bytes, 8));
    if (bytes) H2_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s));
    return d;
  };
  C.rowptr = (int*)up(H.rowptr.data(), sizeof(int) * H.rowptr.size());
  C.col = (int*)up(H.col.data(), sizeof(int) * H.col.size());
  C.blk = (const float**)up(H.blk.data(), sizeof(void*) * H.blk.size());
  C.mode = (unsigned char*)up(H.mode.data(), H.mode.size());
  H2_CUDA(cudaStreamSynchronize(s));   // the host vectors go out of scope
  return C;
}

// Both triangles of a symmetric operator stored by its upper triangle (FP32 copy):
// entry (t, s) is read by rows in row t and by columns in row s.
PanelCSR full_list(Matrix& M, const SymOp& op) {
  std::vector<int> rp(op.nrows + 1), cl(op.nnz);
  std::vector<const float*> bp(op.nnz);
  cudaStream_t s = M.stream;
  H2_CUDA(cudaMemcpyAsync(rp.data(), op.rowptr, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost, s));
  if (op.nnz) {
    H2_CUDA(cudaMemcpyAsync(cl.data(), op.col, sizeof(int) * cl.size(), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaMemcpyAsync(bp.data(), op.blk32, sizeof(void*) * bp.size(), cudaMemcpyDeviceToHost, s));
  }
  H2_CUDA(cudaStreamSynchronize(s));
  std::vector<int> cnt(op.nrows + 1, 0);
  for (int t = 0; t < op.nrows; ++t)
    for (int e = rp[t]; e < rp[t + 1]; ++e) {
      cnt[t + 1]++;
      if (cl[e] != t) cnt[cl[e] + 1]++;
    }
  for (int t = 0; t < op.nrows; ++t) cnt[t + 1] += cnt[t];
  HostList H;
  H.rowptr.assign(cnt.begin(), cnt.end());
  H.col.resize(cnt.back());
  H.blk.resize(cnt.back());
  H.mode.resize(cnt.back());
  std::vector<int> pos(cnt.begin(), cnt.end() - 1);
  for (int t = 0; t < op.nrows; ++t)
    for (int e = rp[t]; e < rp[t + 1]; ++e) {
      const int sc = cl[e];
      int k = pos[t]++;
      H.col[k] = sc;
      H.blk[k] = bp[e];
      H.mode[k] = BM_ROW;
      if (sc != t) {
        k = pos[sc]++;
        H.col[k] = t;
        H.blk[k] = bp[e];
        H.mode[k] = BM_COL;
      }
    }
  return upload_list(M, H);
}

void build_plan(Matrix& M) {
  const int L = M.L, ts = M.tstar;
  const int nleaf = 1 << L;
  auto* P = new PanelPlan();
  M.panel = P;
  const size_t panel = (size_t)PW * PK;
  P->xp = (char*)M.alloc((size_t)kPanelSP * nleaf);
  P->yp = (float*)M.alloc(sizeof(float) * panel * nleaf);
  P->near = full_list(M, M.opD);
  HostList fin;
  if (ts >= 0) {
    const size_t ns = (size_t)M.nslots();
    P->xc = (char*)M.alloc((size_t)kPanelSP * ns);
    P->yr = (float*)M.alloc(sizeof(float) * panel * ns);
    P->yc = (char*)M.alloc((size_t)kPanelSP * ns);
    P->coup = full_list(M, M.opC[1]);
    const size_t kk = (size_t)PK * PK;
    HostList lu;   // x_hat_l = U_l^T x_l: column b of U_l (column-major) is operand row b
    for (int l = 0; l < nleaf; ++l) {
      lu.add(l, M.d_U32 + (size_t)l * kk, BM_NAT);
      lu.end_row();
      fin.add(M.slot0(L) + l, M.d_UT32 + (size_t)l * kk, BM_NAT);   // y_l += U_l y_hat_l (rows of U_l)
      fin.end_row();
    }
    P->lup = upload_list(M, lu);
    P->up.assign(L + 1, PanelCSR{});
    P->down.assign(L + 1, PanelCSR{});
    for (int ell = L; ell > ts; --ell) {   // parents at ell - 1 from children at ell (E_c^T)
      HostList H;
      for (int p = 0; p < (1 << (ell - 1)); ++p) {
        for (int c = 2 * p; c < 2 * p + 2; ++c) H.add(M.slot0(ell) + c, M.d_E32 + (size_t)(M.slot0(ell) + c) * kk, BM_NAT);
        H.end_row();
      }
      P->up[ell] = upload_list(M, H);
    }
    for (int ell = ts; ell <= L; ++ell) {  // y_hat_c = y_row_c + E_c y_hat_parent (rows of E_c)
      HostList H;
      for (int c = 0; c < (1 << ell); ++c) {
        if (ell > ts) H.add(M.slot0(ell - 1) + c / 2, M.d_ET32 + (size_t)(M.slot0(ell) + c) * kk, BM_NAT);
        H.end_row();
      }
      P->down[ell] = upload_list(M, H);
    }
  } else {
    for (int l = 0; l < nleaf; ++l) fin.end_row();
  }
  P->lfin = upload_list(M, fin);
}

void launch(Matrix& M, const PanelCSR& C, const char* xin, const float* cin, int64_t cin_off, void* out,
            bool out_split, int64_t out_off, double* y, int64_t ldy, int nr, cudaStream_t s) {
  if (C.nrows == 0) return;
  PanelArgs a{};
  a.rowptr = C.rowptr;
  a.col = C.col;
  a.blk = C.blk;
  a.mode = C.mode;
  a.xin = xin;
  a.cin = cin;
  a.out = out;
  a.out_split = out_split ? 1 : 0;
  a.cin_off = cin_off;
  a.out_off = out_off;
  a.leafoff = M.d_leafoff;
  a.perm = M.d_perm;
  a.y = y;
  a.ldy = ldy;
  a.nr = nr;
  a.flag = M.d_flag + 1;
  { k_panel_mma<<<C.nrows, 256, kDynSmem, s>>>(a); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
}

}  // namespace

int64_t panel_entries(const Matrix& M) {
  if (!M.panel) return 0;
  const PanelPlan& P = *M.panel;
  int64_t v = P.lup.nnz + P.near.nnz + P.coup.nnz + P.lfin.nnz;
  for (auto& c : P.up) v += c.nnz;
  for (auto& c : P.down) v += c.nnz;
  return v;
}

bool panel_supported(const Matrix& M) { return M.with_f32 && M.KD == PK && (M.tstar < 0 || M.KC == PK); }

// Y = A X (level 1) for nr columns through the tensor cores, 128 columns per pass.
void apply_panel(Matrix& M, const double* x, int64_t ldx, double* y, int64_t ldy, int nr, cudaStream_t s) {
  H2_REQUIRE(M.with_f32, H2MG_ERR_INVALID_ARG, "the tensor-core product needs the FP32 copy (with_f32)");
  H2_REQUIRE(panel_supported(M), H2MG_ERR_UNSUPPORTED, "the tensor-core product needs leaf and rank blocks of 64");
  H2_CUDA(cudaFuncSetAttribute(k_panel_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem));
  if (!M.panel) build_plan(M);
  PanelPlan& P = *M.panel;
  const int L = M.L, ts = M.tstar, nleaf = 1 << L;
  H2_CUDA(cudaMemsetAsync(M.d_flag + 1, 0, sizeof(int), s));
  for (int c0 = 0; c0 < nr; c0 += PW) {
    const int g = std::min(PW, nr - c0);
    const int64_t tot = (int64_t)nleaf * PW * PK;
    { k_panel_in<<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(x + (int64_t)c0 * ldx, ldx, g, M.d_leafoff, M.d_perm,
                                                               nleaf, P.xp); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    if (ts >= 0) {
      launch(M, P.lup, P.xp, nullptr, 0, P.xc, true, M.slot0(L), nullptr, 0, 0, s);
      for (int ell = L; ell > ts; --ell)
        launch(M, P.up[ell], P.xc, nullptr, 0, P.xc, true, M.slot0(ell - 1), nullptr, 0, 0, s);
    }
    launch(M, P.near, P.xp, nullptr, 0, P.yp, false, 0, nullptr, 0, 0, s);
    if (ts >= 0) {
      launch(M, P.coup, P.xc, nullptr, 0, P.yr, false, 0, nullptr, 0, 0, s);
      for (int ell = ts; ell <= L; ++ell)
        launch(M, P.down[ell], P.yc, P.yr, M.slot0(ell), P.yc, true, M.slot0(ell), nullptr, 0, 0, s);
    }
    launch(M, P.lfin, ts >= 0 ? P.yc : P.xp, P.yp, 0, nullptr, false, 0, y + (int64_t)c0 * ldy, ldy, g, s);
  }
  int h = 0;
  H2_CUDA(cudaMemcpyAsync(&h, M.d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
  H2_REQUIRE(h == 0, H2MG_ERR_CUDA, "a tensor-core product timed out waiting for its MMAs");
}

}  // namespace h2mg
