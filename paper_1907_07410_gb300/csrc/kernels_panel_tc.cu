// Panel products of the eigen-solver on the tcgen05 tensor cores:
//   out = alpha G in + beta in + gamma in2
// for one 128-row tile of one block's Gram matrix G (s_pad x s_pad, float32,
// symmetric) and its b-column panel `in` (s_pad x b, row-major).
//
// Precision: three tf32 products. Every float32 operand x is split into
// hi = x rounded to 10 mantissa bits (exact in tf32) and lo = x - hi
// (exact in float32, |lo| <= 2^-11 |x|), and
//   G in ~= G_hi in_hi + G_hi in_lo + G_lo in_hi.
// The dropped G_lo in_lo term and the tf32 narrowing of the lo parts are
// below 2^-21 relative. Splitting explicitly (rather than leaving the low
// bits to the MMA) makes the result independent of how the hardware narrows
// f32 to tf32.
//
// The panel operand is read in "B form": for each 32-row chunk of `in`,
// b rows of hi (one per panel column, its 32 values of that chunk), then b
// rows of lo, 32 floats each (s_pad x 2b floats per block). It is K-major,
// as the MMA's B operand must be, and the split is done once per panel
// rather than once per 128-row tile of G. The epilogue writes the B form of
// `out` next to it (when asked), so each product feeds the next; launch_bform
// converts a panel written by another kernel.
//
// Data path, per stage of 64 floats of K:
//   * TMA loads of the G tile (128 rows x 64 floats, as two 32-float boxes)
//     and the two matching B-form chunks (2b rows x 32 floats each), all
//     with 128-byte swizzling. The panel products keep them in two rings,
//     each with its own producer warp (warp 0 for G, warp 14 for the B
//     form), and release a G stage as soon as the converters have read it;
//     the projection loads both into one ring from warp 0;
//   * warps 2-9 (converters, two per TMEM lane quarter, one per 32-float
//     half of the stage): each thread reads one row of its half of the G
//     tile, splits it in registers and stores hi and lo into a
//     tensor-memory slot (tcgen05.st; lane = row, one column per K
//     element), the A operand layout of kind::tf32. The tensor core reads
//     shared memory at 128 bytes per cycle, so an A operand read from
//     shared memory (4 KiB per K = 8) would cost 32 cycles per MMA;
//   * warp 1: per K = 8 slice, two MMAs with A in tensor memory:
//     G_hi x [in_hi | in_lo] (N = 2b) and G_lo x in_hi (N = b). The first
//     gives the main product and one cross term side by side; the second adds
//     the other cross term onto the first's cross half.
//   * warps 10-13 (the products' epilogue, one per TMEM lane quarter): read
//     a tile's accumulators into registers and release them at once, then
//     apply the Chebyshev step and write `out` while the next tile's MMAs
//     run. (When the converter warps ran the epilogue as well, the MMA warp
//     waited for it about 300 cycles per stage on the 480,189 x 17,770
//     workload, and the products ran at 0.74 of HBM; 0.79 with these
//     warps, 0.82 with the two rings, 0.83 with three G stages and four B
//     stages at b = 64: measured against four and three, five and two,
//     and two and five, the B ring's depth mattered more.)
// Warps 0 and 1 run their loops as whole warps, so addresses and
// descriptors stay warp-uniform, and one elected lane issues. Measured on
// GB300 (clock stamps per stage), a single lane running the same loop took
// about 90 cycles per MMA and 300 more per satisfied barrier wait; now a
// stage's 16 MMAs issue in about 400 cycles. Eight converter warps (four
// took about 1000 cycles per stage) bring the kernel to about 740 cycles
// per 32 floats of K on a 988-row block.
//
// Launch: programmatic dependent launch. A product's prologue (tile, state,
// barriers, tensor memory) overlaps the end of the previous kernel, and
// griddepcontrol.wait precedes every read of a panel and every write of
// `out`. The epilogue reads in, in2 and writes out with 16-byte accesses (a
// thread owns a row). Back to back, 16 blocks of 988 rows take 12.4 us per
// product (18.6 us with plain launches, scalar epilogue accesses and four
// converter warps).
//
// Accumulation: the tensor core's f32 accumulator does not round to
// nearest at each step (a measured one-signed error growing with the number
// of accumulating MMAs), so long chains drift: one accumulator over the
// whole K range of a 1000-row block gave errors near 1e-5 relative. The K
// slices therefore go round-robin into R accumulators (4, or 2 for b = 64,
// as tensor memory allows) and the epilogue adds them in a fixed order,
// main halves and cross halves separately, then the two sums.
//
// Tensor memory (512 columns): R accumulators of 2b columns, then kSlots
// (2) slots of 128 columns (64 hi, 64 lo) for the A operand.
//
// Every wait is bounded; a timeout sets kErrTimeout and the CTA drains its
// copies in flight and frees its tensor memory before returning.
//
// The projection F_L = W^T F_s (k_project_tc, with k_bform_fs for F_s's B
// form) reuses this data path; see its comment below.
#include <type_traits>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace bsvd {

namespace {

constexpr int PT = 128;                  // G rows per CTA (MMA M)
constexpr int PK = 64;                   // floats of K per stage
constexpr int PH = 32;                   // floats per 128-byte swizzle row
constexpr int kThreads = 320;            // 10 warps (projection)
constexpr int kPConv = 8;                // panel products: converter warps
constexpr int kBWarp = 2 + kPConv + 4;   // their B-stage producer warp
constexpr int kPThreads = 32 * (kBWarp + 1);  // 15 warps
constexpr int kMaxGS = 6, kMaxBS = 4;    // the products' G and B rings
constexpr int kConv = 8;                 // converter warps (2..9)
constexpr int kMaxStages = 4;
constexpr int kSlots = 2;                // A slots in tensor memory
constexpr uint32_t kSpinP = 1u << 22;    // mbarrier polls before giving up
constexpr int G_HALF = PT * PH * 4;      // 16 KiB: one 32-float box of G
constexpr int G_BYTES = 2 * G_HALF;
constexpr int kTmemCols = 512;

template <int B>
struct PanelTc {
  static constexpr int BOP_HALF = 2 * B * 128;      // one B-form chunk
  static constexpr int BOP_BYTES = 2 * BOP_HALF;
  static constexpr int STAGE = G_BYTES + BOP_BYTES;
  static constexpr int STAGES = B >= 64 ? 3 : 4;
  static constexpr int R = B >= 64 ? 2 : 4;          // accumulators
  static constexpr int ACC_COLS = R * 2 * B;
  static constexpr bool kWaitSlot = kSlots < STAGES; // else implied by `empty`
  static_assert(STAGE % 1024 == 0, "stage regions stay 1024-byte aligned");
  static_assert(ACC_COLS + kSlots * 2 * PK <= kTmemCols, "tensor memory");
  static_assert(STAGES <= kMaxStages && STAGES >= kSlots, "ring sizes");
};

constexpr int kTq = 4;                   // tile-index ring of the products

struct PanelCtrl {
  uint64_t full[kMaxStages];    // G tile and rows of `in` landed (TMA bytes)
  uint64_t empty[kMaxStages];   // the stage's MMAs completed
  uint64_t ready[kSlots];       // A slot written (the 8 converter warps)
  uint64_t afree[kSlots];       // the MMAs reading the A slot completed
  uint64_t done;                // a tile's MMAs completed (one phase a tile)
  uint64_t accfree;             // the epilogue read the accumulators (4 warps)
  uint64_t tfull[kTq];          // tile index published (the producer)
  uint64_t tempty[kTq];         // tile index read (warps 1-9)
  int tq[kTq];                  // tile indices, -1 ends the launch
  uint32_t tmem;
  int abort;
  int issued;                   // stages whose loads were issued
  int consumed;                 // stages the A converters saw land
};

template <int B>
constexpr size_t panel_tc_smem() {
  return PanelTc<B>::STAGES * PanelTc<B>::STAGE + sizeof(PanelCtrl) + 1024;
}

__device__ __forceinline__ float hi1(float x) { return tf32_hi(x); }

__device__ __forceinline__ float4 hi4(float4 v) {
  return make_float4(hi1(v.x), hi1(v.y), hi1(v.z), hi1(v.w));
}

__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
  return make_float4(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y),
                     __fsub_rn(a.z, b.z), __fsub_rn(a.w, b.w));
}

// Byte offset of the 16-byte chunk `c` (0..7) of row `r` in a tile of
// 128-byte rows stored with 128-byte swizzling (tile base 1024-aligned).
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

// Sum of the R accumulators' 16 columns at `col`, in a fixed order:
// (a0 + a1) + (a2 + a3), or a0 + a1.
template <int B>
__device__ __forceinline__ void acc_sum(uint32_t taddr, uint32_t col,
                                        float (&v)[16]) {
  using L = PanelTc<B>;
  float t[16];
  tc::tmem_ld16(taddr + col, v);
  tc::tmem_ld16(taddr + col + 2 * B, t);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] += t[j];
  if constexpr (L::R == 4) {
    float u[16];
    tc::tmem_ld16(taddr + col + 4 * B, u);
    tc::tmem_ld16(taddr + col + 6 * B, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] += u[j] + t[j];
  }
}

// A converter thread's hi or lo values into its TMEM lane (32 columns)
__device__ __forceinline__ void tmem_st_row(uint32_t ta, const float (&v)[32]) {
  tc::tmem_st32(ta, v);
}

// True when tile `t`'s block takes part in this product: still iterating,
// and (for a filter step) its own filter reaches this step.
__device__ __forceinline__ bool tile_active(const SolverState *state, int2 t,
                                            int mode, int step) {
  const SolverState &st = state[t.x];
  return st.status == kRunning && !(mode >= 1 && step > st.degree);
}

// The persistent products keep G and the panel's B form in separate rings.
// A G stage (128 rows x 64 floats, from HBM) is released as soon as the
// converter warps have read it into registers, before its MMAs run; a B
// stage (from L2: every row tile of a block reads the same panel) when its
// MMAs complete. Each ring has its own producer warp, so G's loads run up to
// GS stages ahead of the conversions whatever the MMAs are doing.
template <int B>
struct PanelRings {
  static constexpr int BOP_HALF = 2 * B * 128;      // one B-form chunk
  static constexpr int BOP_BYTES = 2 * BOP_HALF;
  static constexpr int GS = B >= 64 ? 3 : (B >= 32 ? 5 : 6);
  static constexpr int BS = 4;
  static constexpr int R = PanelTc<B>::R;
  static constexpr int ACC_COLS = PanelTc<B>::ACC_COLS;
  static constexpr int B_OFF = GS * G_BYTES;         // the B ring follows G's
  static constexpr int RINGS = B_OFF + BS * BOP_BYTES;
  static_assert(BOP_BYTES % 1024 == 0, "stage regions stay 1024-byte aligned");
  static_assert(GS <= kMaxGS && BS <= kMaxBS && BS >= 2, "ring sizes");
};

struct PanelRingCtrl {
  uint64_t gfull[kMaxGS];       // G stage landed (TMA bytes)
  uint64_t gempty[kMaxGS];      // G stage read by the converter warps
  uint64_t bfull[kMaxBS];       // B stage landed (TMA bytes)
  uint64_t bempty[kMaxBS];      // the B stage's MMAs completed
  uint64_t ready[kSlots];       // A slot written (the converter warps)
  uint64_t afree[kSlots];       // the MMAs reading the A slot completed
  uint64_t done;                // a tile's MMAs completed (one phase a tile)
  uint64_t accfree;             // the epilogue read the accumulators (4 warps)
  uint64_t tfull[kTq];          // tile index published (warp 0)
  uint64_t tempty[kTq];         // tile index read (the other warps)
  int tq[kTq];                  // tile indices, -1 ends the launch
  uint32_t tmem;
  int abort;
  int gissued, gconsumed;       // G stages issued / seen to land
  int bissued, bconsumed;       // B stages issued / seen to land
};

template <int B>
constexpr size_t panel_ring_smem() {
  return PanelRings<B>::RINGS + sizeof(PanelRingCtrl) + 1024;
}

// Persistent: one CTA per SM. CTA i starts with tile i (if its block is
// still iterating), then takes tiles from gridDim.x on from a shared
// counter (ctl[0]; ctl[1] counts finished CTAs, and the last one resets
// both for the next launch). A claimed tile of an idle block moves the
// counter past the rest of that block. Warp 0 claims tiles, publishes their
// indices in a small ring (tq) and loads their G stages; warp kBWarp loads
// the matching B stages; warps 2 + kPConv .. + 3 run the epilogue. The stage, A-slot and tile counters run on across
// tiles, so a CTA sets up its barriers and tensor memory once per launch
// and the loads of the next tile overlap the epilogue of the last. The MMA
// warp starts a tile only after the epilogue warps have read the previous
// tile's accumulators (accfree).
template <int B>
__global__ void __launch_bounds__(kPThreads, 1)
k_gpanel_tc(const BlockMeta *__restrict__ meta, SolverState *state,
            const int2 *__restrict__ tiles, int ntiles, int *ctl,
            unsigned long long *ptime, const CUtensorMap *__restrict__ gmaps,
            const CUtensorMap *__restrict__ xmaps, const float *in,
            const float *in2, float *out, float *out_bf, int mode, int step,
            int32_t *err) {
  using L = PanelRings<B>;
  constexpr int GS = L::GS, BS = L::BS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  PanelRingCtrl &ct = *reinterpret_cast<PanelRingCtrl *>(base + L::RINGS);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  auto g_tile = [&](int s) { return base + s * G_BYTES; };
  auto b_op = [&](int s) { return base + L::B_OFF + s * L::BOP_BYTES; };

  if (warp == 0) tc::tmem_alloc(&ct.tmem, kTmemCols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < GS; ++s) {
      tc::mbar_init(&ct.gfull[s], 1);
      tc::mbar_init(&ct.gempty[s], kPConv);
    }
    for (int s = 0; s < BS; ++s) {
      tc::mbar_init(&ct.bfull[s], 1);
      tc::mbar_init(&ct.bempty[s], 1);
    }
    for (int a = 0; a < kSlots; ++a) {
      tc::mbar_init(&ct.ready[a], kPConv);
      tc::mbar_init(&ct.afree[a], 1);
    }
    for (int q = 0; q < kTq; ++q) {
      tc::mbar_init(&ct.tfull[q], 1);
      tc::mbar_init(&ct.tempty[q], 6 + kPConv);  // MMA, converters, epilogue, B loads
    }
    tc::mbar_init(&ct.done, 1);
    tc::mbar_init(&ct.accfree, 4);
    ct.abort = 0;
    ct.gissued = ct.gconsumed = 0;
    ct.bissued = ct.bconsumed = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // everything below reads what the previous kernels wrote: the solver
  // state (which blocks run), the panels and the tile counter's reset
  pdl_wait();
  if (threadIdx.x == 0) atomicMin(&ptime[1], globaltimer_ns());
  const uint32_t taddr = ct.tmem;
  const uint32_t aslots = taddr + L::ACC_COLS;    // A slot a at +128 a
  volatile int *abort_flag = &ct.abort;

  auto give_up = [&]() {
    if (lane == 0) atomicOr(err, kErrTimeout);
    ct.abort = 1;
  };
  // the warps other than 0: the next tile index from the ring, -1 at the end
  auto next_tile = [&](int &got, int &idx) -> bool {
    const int q = got % kTq;
    const bool ok = __all_sync(
        0xffffffffu,
        tc::mbar_wait(&ct.tfull[q], (got / kTq) & 1, kSpinP) && !*abort_flag);
    if (!ok) {
      give_up();
      return false;
    }
    idx = *reinterpret_cast<volatile int *>(&ct.tq[q]);
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&ct.tempty[q]);
    ++got;
    return idx >= 0;
  };

  if (warp == 0) {
    // tiles and G stages; the whole warp runs the loop (warp-uniform
    // addresses) and one lane issues
    int g = 0, pub = 0;
    const int first = (int)gridDim.x;     // tiles below this: one per CTA
    for (;;) {
      int idx = -1;
      if (lane == 0) {
        // the CTA's own tile first, with no atomic; then the counter, which
        // numbers the tiles from gridDim.x on
        if (pub == 0 && (int)blockIdx.x < ntiles &&
            tile_active(state, tiles[blockIdx.x], mode, step)) {
          idx = (int)blockIdx.x;
        } else {
          for (;;) {
            const int i = first + atomicAdd(&ctl[0], 1);
            if (i >= ntiles) break;
            const int2 ti = tiles[i];
            if (tile_active(state, ti, mode, step)) { idx = i; break; }
            // the block is idle: move the counter past its other tiles (a
            // block's tiles are consecutive in the list)
            const BlockMeta &bx = meta[ti.x];
            atomicMax(&ctl[0], bx.pt0 + bx.npt - first);
          }
        }
      }
      idx = __shfl_sync(0xffffffffu, idx, 0);
      const int q = pub % kTq;
      bool ok = __all_sync(0xffffffffu,
                           tc::mbar_wait(&ct.tempty[q], ((pub / kTq) & 1) ^ 1,
                                         kSpinP) && !*abort_flag);
      if (!ok) {
        give_up();
        break;
      }
      if (lane == 0) {
        ct.tq[q] = idx;
        tc::mbar_arrive(&ct.tfull[q]);
      }
      __syncwarp();
      ++pub;
      if (idx < 0) break;
      const int2 t = tiles[idx];
      const BlockMeta bm = meta[t.x];
      if (t.y == 0 && lane == 0) atomicAdd(&state[t.x].products, 1);
      // s_pad is a multiple of 32: a last half stage reads zeros past s_pad
      const int nk = (bm.s_pad + PK - 1) / PK;
      const CUtensorMap *map = gmaps + t.x;
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = g % GS;
        ok = __all_sync(0xffffffffu,
                        tc::mbar_wait(&ct.gempty[s], ((g / GS) & 1) ^ 1,
                                      kSpinP) && !*abort_flag);
        if (!ok) {
          give_up();
          break;
        }
        if (tc::elect_one()) {
          const int k0 = kc * PK;
          tc::mbar_expect_tx(&ct.gfull[s], G_BYTES);
          tc::tma_load_2d(g_tile(s), map, k0, t.y, &ct.gfull[s]);
          tc::tma_load_2d(g_tile(s) + G_HALF, map, k0 + PH, t.y, &ct.gfull[s]);
          ct.gissued = g + 1;
        }
        __syncwarp();
      }
      if (!ok) break;
    }
  } else if (warp == kBWarp) {
    // B stages: the B-form chunks 2 kc and 2 kc + 1 of the tile's panel
    // (past the last: zero fill)
    int got = 0, idx = -1, gb = 0;
    while (next_tile(got, idx)) {
      const int2 t = tiles[idx];
      const BlockMeta bm = meta[t.x];
      const int nk = (bm.s_pad + PK - 1) / PK;
      const CUtensorMap *xmap = xmaps + t.x;
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc, ++gb) {
        const int s = gb % BS;
        ok = __all_sync(0xffffffffu,
                        tc::mbar_wait(&ct.bempty[s], ((gb / BS) & 1) ^ 1,
                                      kSpinP) && !*abort_flag);
        if (!ok) break;
        if (tc::elect_one()) {
          tc::mbar_expect_tx(&ct.bfull[s], L::BOP_BYTES);
          tc::tma_load_2d(b_op(s), xmap, 0, 2 * kc * 2 * B, &ct.bfull[s]);
          tc::tma_load_2d(b_op(s) + L::BOP_HALF, xmap, 0,
                          (2 * kc + 1) * 2 * B, &ct.bfull[s]);
          ct.bissued = gb + 1;
        }
        __syncwarp();
      }
      if (!ok) {
        give_up();
        break;
      }
    }
  } else if (warp == 1) {
    // the whole warp runs the loop (warp-uniform descriptors); one lane issues
    constexpr uint32_t idesc2 = tc::idesc_tf32_f32(PT, 2 * B);
    constexpr uint32_t idesc1 = tc::idesc_tf32_f32(PT, B);
    int got = 0, idx = -1, gm = 0, tl = 0;
    while (next_tile(got, idx)) {
      const BlockMeta bm = meta[tiles[idx].x];
      const int nk = (bm.s_pad + PK - 1) / PK;
      bool ok = true;
      if (tl > 0) {
        // the previous tile's accumulators have been read
        ok = __all_sync(0xffffffffu,
                        tc::mbar_wait(&ct.accfree, (tl - 1) & 1, kSpinP) &&
                            !*abort_flag);
      }
      for (int kc = 0; ok && kc < nk; ++kc, ++gm) {
        const int s = gm % BS, a = gm % kSlots;
        ok = __all_sync(
            0xffffffffu,
            tc::mbar_wait(&ct.bfull[s], (gm / BS) & 1, kSpinP) &&
                tc::mbar_wait(&ct.ready[a], (gm / kSlots) & 1, kSpinP) &&
                !*abort_flag);
        if (!ok) break;
        if (lane == 0) ct.bconsumed = gm + 1;
        tc::fence_after_sync();
        const uint64_t db0 = tc::sdesc_kmajor_sw128(tc::smem_u32(b_op(s)));
        const uint64_t db1 =
            tc::sdesc_kmajor_sw128(tc::smem_u32(b_op(s) + L::BOP_HALF));
        const uint32_t ahi = aslots + 2 * PK * a, alo = ahi + PK;
        if (tc::elect_one()) {
          // K slice 8 kc + kk goes to accumulator kk mod R; the first R
          // slices of a tile start their accumulators
#pragma unroll
          for (int kk = 0; kk < PK / 8; ++kk) {
            const uint32_t d = taddr + 2 * B * (kk % L::R);
            const uint64_t db = (kk < 4 ? db0 : db1) + 2 * (kk & 3);
            const uint32_t acc = (kc > 0 || kk >= L::R) ? 1u : 0u;
            // [G_hi in_hi | G_hi in_lo], then G_lo in_hi onto the cross half
            tc::mma_tf32_ta(d, ahi + 8 * kk, db, idesc2, acc);
            tc::mma_tf32_ta(d + B, alo + 8 * kk, db, idesc1, 1u);
          }
          tc::mma_commit(&ct.bempty[s]);
          tc::mma_commit(&ct.afree[a]);
        }
        __syncwarp();
      }
      if (!ok) {
        give_up();
        break;
      }
      if (tc::elect_one()) tc::mma_commit(&ct.done);
      __syncwarp();
      ++tl;
    }
  } else if (warp < 2 + kPConv) {
    // converters: warps 2 .. 2 + kPConv - 1. Warp w may touch TMEM lanes
    // 32 (w mod 4) .. +31, so kPConv / 4 warps share each lane quarter, one
    // per CF-float part kq of a stage's 64-float K range (warps 2-5 kq = 0,
    // 6-9 kq = 1, ...).
    constexpr int CF = 4 * PK / kPConv;           // floats per converter
    const int cid = threadIdx.x - 64;
    const int q = warp & 3;
    const int kq = (warp - 2) >> 2;
    const int r = q * 32 + lane;                  // G tile row of this thread
    const uint32_t lrow = (uint32_t)(q * 32) << 16;
    int got = 0, idx = -1, gc = 0, tl = 0;
    while (next_tile(got, idx)) {
      const int2 t = tiles[idx];
      const BlockMeta bm = meta[t.x];
      const int nk = (bm.s_pad + PK - 1) / PK;
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc, ++gc) {
        const int s = gc % GS, a = gc % kSlots;
        // warp-uniform: every lane breaks, or none does
        ok = __all_sync(0xffffffffu,
                        tc::mbar_wait(&ct.gfull[s], (gc / GS) & 1, kSpinP) &&
                            !*abort_flag);
        if (!ok) break;
        if (cid == 0) ct.gconsumed = gc + 1;
        tc::fence_after_sync();
        // this thread's row of its part of the G tile (CF floats of the
        // 32-float box kq CF / 32, from chunk (kq CF mod 32) / 4), split
        // into hi and lo
        float h[CF], l[CF];
        {
          const unsigned char *gt = g_tile(s) + ((kq * CF) / PH) * G_HALF;
          const int c0 = ((kq * CF) % PH) / 4;
#pragma unroll
          for (int c = 0; c < CF / 4; ++c) {
            const float4 v =
                *reinterpret_cast<const float4 *>(gt + sw128(r, c0 + c));
            const float4 vh = hi4(v), vl = sub4(v, vh);
            h[4 * c + 0] = vh.x; h[4 * c + 1] = vh.y;
            h[4 * c + 2] = vh.z; h[4 * c + 3] = vh.w;
            l[4 * c + 0] = vl.x; l[4 * c + 1] = vl.y;
            l[4 * c + 2] = vl.z; l[4 * c + 3] = vl.w;
          }
        }
        // the stage's values are in registers: release it to the G loads
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&ct.gempty[s]);
        // the A slot's previous MMAs have completed
        ok = __all_sync(0xffffffffu,
                        tc::mbar_wait(&ct.afree[a], ((gc / kSlots) & 1) ^ 1,
                                      kSpinP) && !*abort_flag);
        if (!ok) break;
        tc::fence_after_sync();
        const uint32_t ta = aslots + lrow + 2 * PK * a + CF * kq;
        tmem_st_row(ta, h);
        tmem_st_row(ta + PK, l);
        tc::tmem_wait_st();
        // order the tensor-memory stores before the MMAs
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&ct.ready[a]);
      }
      if (!ok) {
        give_up();
        break;
      }
      ++tl;
    }
  } else {
    // the epilogue: warps 10-13, one per TMEM lane quarter (warp mod 4).
    // A tile's accumulators are read into registers (main and cross halves
    // added) and released at once, so the MMAs of the next tile can start
    // while these warps read in, in2 and write out.
    const int q = warp & 3;
    const int r = q * 32 + lane;                  // G tile row of this thread
    const uint32_t lrow = (uint32_t)(q * 32) << 16;
    int got = 0, idx = -1, tl = 0;
    while (next_tile(got, idx)) {
      const int2 t = tiles[idx];
      const BlockMeta bm = meta[t.x];
      bool ok = __all_sync(0xffffffffu,
                           tc::mbar_wait(&ct.done, tl & 1, kSpinP) &&
                               !*abort_flag);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      tc::fence_after_sync();
      float acc[B];
#pragma unroll
      for (int c0 = 0; c0 < B; c0 += 16) {
        float v[16], w[16];
        acc_sum<B>(taddr + lrow, c0, v);        // main halves
        acc_sum<B>(taddr + lrow, B + c0, w);    // cross halves
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[c0 + u] = v[u] + w[u];
      }
      // the accumulators may be overwritten by the next tile's MMAs
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&ct.accfree);
      const SolverState st = state[t.x];
      float alpha, beta, gamma;
      cheb_coeffs(st, mode, step, &alpha, &beta, &gamma);
      const int rr = t.y + r;                    // output row
      if (rr < bm.s_pad) {
        const float *inb = in + bm.x_off;
        const float *in2b = in2 ? in2 + bm.x_off : nullptr;
        float *outb = out + bm.x_off;
        // B form of `out`: chunk rr / 32, position rr mod 32 (lanes of a
        // warp hold 32 consecutive rows of one chunk: coalesced 128 bytes)
        float *bfb = out_bf ? out_bf + 2 * bm.x_off +
                                  (int64_t)(rr >> 5) * 2 * B * 32 + (rr & 31)
                            : nullptr;
        // a thread's row of `out` (and of in, in2) is contiguous: 16-byte
        // accesses, 4 columns each
        const int64_t o0 = (int64_t)rr * B;
#pragma unroll
        for (int c4 = 0; c4 < B / 4; ++c4) {
          float y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) y[u] = alpha * acc[4 * c4 + u];
          if (beta != 0.f) {
            const float4 x = *reinterpret_cast<const float4 *>(inb + o0 + 4 * c4);
            y[0] = fmaf(beta, x.x, y[0]); y[1] = fmaf(beta, x.y, y[1]);
            y[2] = fmaf(beta, x.z, y[2]); y[3] = fmaf(beta, x.w, y[3]);
          }
          if (gamma != 0.f) {
            const float4 x = *reinterpret_cast<const float4 *>(in2b + o0 + 4 * c4);
            y[0] = fmaf(gamma, x.x, y[0]); y[1] = fmaf(gamma, x.y, y[1]);
            y[2] = fmaf(gamma, x.z, y[2]); y[3] = fmaf(gamma, x.w, y[3]);
          }
          *reinterpret_cast<float4 *>(outb + o0 + 4 * c4) =
              make_float4(y[0], y[1], y[2], y[3]);
          if (bfb) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c = 4 * c4 + u;
              const float yh = hi1(y[u]);
              bfb[c * 32] = yh;
              bfb[(B + c) * 32] = __fsub_rn(y[u], yh);
            }
          }
        }
      }
      ++tl;
    }
  }
  __syncwarp();
  // the next kernel may be scheduled now; it waits for this grid to
  // complete before it reads a panel
  pdl_trigger();
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && ct.abort) {
    // drain stages that were issued but never seen to land
    for (int g = ct.gconsumed; g < ct.gissued; ++g)
      tc::mbar_wait(&ct.gfull[g % GS], (g / GS) & 1, kSpinP);
    for (int g = ct.bconsumed; g < ct.bissued; ++g)
      tc::mbar_wait(&ct.bfull[g % BS], (g / BS) & 1, kSpinP);
  }
  if (threadIdx.x == 0) {
    // the last CTA out resets the tile counter for the next launch
    __threadfence();
    if (atomicAdd(&ctl[1], 1) == (int)gridDim.x - 1) {
      // and adds this launch's span (first start to last end) to ptime[0]
      // (the two dies' timers may differ by a little: a negative span of a
      // very short launch counts as 0)
      const unsigned long long t0 = atomicAdd(&ptime[1], 0ull);
      const unsigned long long t1 = globaltimer_ns();
      if (t1 > t0 && t0 != ~0ull) atomicAdd(&ptime[0], t1 - t0);
      atomicAdd(&ptime[2], 1ull);          // launches
      atomicExch(&ptime[1], ~0ull);
      atomicExch(&ctl[0], 0);
      atomicExch(&ctl[1], 0);
      __threadfence();
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

template <int B>
cudaError_t launch_b(const BlockMeta *meta, SolverState *state,
                     const int2 *tiles, int32_t ntiles, int32_t nctas, int *ctl,
                     unsigned long long *ptime,
                     const CUtensorMap *gmaps, const CUtensorMap *xmaps,
                     const float *in, const float *in2, float *out,
                     float *out_bf, int mode, int step, int32_t *err,
                     cudaStream_t st) {
  static_assert(panel_ring_smem<B>() <= 227 * 1024, "shared memory");
  cudaError_t e = cudaFuncSetAttribute(
      k_gpanel_tc<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)panel_ring_smem<B>());
  if (e != cudaSuccess) return e;
  // programmatic dependent launch: this grid's prologue may overlap the end
  // of the previous kernel in the stream (see pdl_wait)
  return launch_pdl(k_gpanel_tc<B>, dim3((unsigned)nctas), dim3(kPThreads),
                    panel_ring_smem<B>(), st, meta, state, tiles, (int)ntiles,
                    ctl, ptime, gmaps, xmaps, in, in2, out, out_bf, mode, step,
                    err);
}

// F_L = W^T F_s on the tensor cores, with the panel product's data path and
// precision (three tf32 products, R accumulators): a CTA computes 128
// consecutive rows l of F_L (columns of W) over the whole K range a < s.
//   * A = the W^T tile: TMA boxes of W of 32 rows a x 128 columns l (plain
//     layout). Converter thread l reads its column (a warp reads 32
//     consecutive l of one row, no bank conflicts), splits it and stores hi
//     and lo to tensor memory, as the panel kernel does with rows of G;
//   * B = F_s in B form (launch_bform_fs), zero past column kp;
//   * epilogue: F_L rows l < L, the kp columns.
template <int B>
__global__ void __launch_bounds__(kThreads, 1)
k_project_tc(const BlockMeta *__restrict__ meta, const int2 *__restrict__ tiles,
             const CUtensorMap *__restrict__ wmaps,
             const CUtensorMap *__restrict__ fmaps, float *FL, int kp,
             int32_t *err) {
  using L = PanelTc<B>;
  constexpr int S = L::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  PanelCtrl &ct = *reinterpret_cast<PanelCtrl *>(base + S * L::STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int l0 = t.y;
  const int nk = (bm.s_pad + PK - 1) / PK;

  auto w_tile = [&](int s) { return base + s * L::STAGE; };
  auto b_op = [&](int s) { return base + s * L::STAGE + G_BYTES; };

  if (warp == 0) tc::tmem_alloc(&ct.tmem, kTmemCols);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&ct.full[s], 1);
      tc::mbar_init(&ct.empty[s], 1);
    }
    for (int a = 0; a < kSlots; ++a) {
      tc::mbar_init(&ct.ready[a], kConv);
      tc::mbar_init(&ct.afree[a], 1);
    }
    tc::mbar_init(&ct.done, 1);
    ct.abort = 0;
    ct.issued = 0;
    ct.consumed = 0;
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // F_s's B form comes from the previous kernel
  pdl_wait();
  const uint32_t taddr = ct.tmem;
  const uint32_t aslots = taddr + L::ACC_COLS;
  volatile int *abort_flag = &ct.abort;

  if (warp == 0) {
    const CUtensorMap *wmap = wmaps + t.x;
    const CUtensorMap *fmap = fmaps + t.x;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % S;
      const uint32_t ph = (kc / S) & 1;
      const bool ok = __all_sync(
          0xffffffffu,
          tc::mbar_wait(&ct.empty[s], ph ^ 1, kSpinP) && !*abort_flag);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      if (tc::elect_one()) {
        const int k0 = kc * PK;
        tc::mbar_expect_tx(&ct.full[s], G_BYTES + L::BOP_BYTES);
        // rows a = k0 .. k0+31 and k0+32 .. k0+63 of W (zero past s_pad)
        tc::tma_load_2d(w_tile(s), wmap, l0, k0, &ct.full[s]);
        tc::tma_load_2d(w_tile(s) + G_HALF, wmap, l0, k0 + PH, &ct.full[s]);
        tc::tma_load_2d(b_op(s), fmap, 0, 2 * kc * 2 * B, &ct.full[s]);
        tc::tma_load_2d(b_op(s) + L::BOP_HALF, fmap, 0, (2 * kc + 1) * 2 * B,
                        &ct.full[s]);
        ct.issued = kc + 1;
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    constexpr uint32_t idesc2 = tc::idesc_tf32_f32(PT, 2 * B);
    constexpr uint32_t idesc1 = tc::idesc_tf32_f32(PT, B);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % S, a = kc % kSlots;
      const bool ok = __all_sync(
          0xffffffffu, tc::mbar_wait(&ct.ready[a], (kc / kSlots) & 1, kSpinP) &&
                           !*abort_flag);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      tc::fence_after_sync();
      const uint64_t db0 = tc::sdesc_kmajor_sw128(tc::smem_u32(b_op(s)));
      const uint64_t db1 =
          tc::sdesc_kmajor_sw128(tc::smem_u32(b_op(s) + L::BOP_HALF));
      const uint32_t ahi = aslots + 2 * PK * a, alo = ahi + PK;
      if (tc::elect_one()) {
#pragma unroll
        for (int kk = 0; kk < PK / 8; ++kk) {
          const uint32_t d = taddr + 2 * B * (kk % L::R);
          const uint64_t db = (kk < 4 ? db0 : db1) + 2 * (kk & 3);
          const uint32_t acc = (kc > 0 || kk >= L::R) ? 1u : 0u;
          tc::mma_tf32_ta(d, ahi + 8 * kk, db, idesc2, acc);
          tc::mma_tf32_ta(d + B, alo + 8 * kk, db, idesc1, 1u);
        }
        tc::mma_commit(&ct.empty[s]);
        tc::mma_commit(&ct.afree[a]);
      }
      __syncwarp();
    }
    if (tc::elect_one()) tc::mma_commit(&ct.done);
    __syncwarp();
  } else {
    // converters (warps 2-9): lane quarter q, K half kh, as in k_gpanel_tc
    const int cid = threadIdx.x - 64;
    const int q = warp & 3;
    const int kh = (warp - 2) >> 2;
    const int r = q * 32 + lane;                  // row l0 + r of F_L
    const uint32_t lrow = (uint32_t)(q * 32) << 16;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % S, a = kc % kSlots;
      const uint32_t ph = (kc / S) & 1;
      bool ok = tc::mbar_wait(&ct.full[s], ph, kSpinP);
      if constexpr (L::kWaitSlot)
        ok = ok && tc::mbar_wait(&ct.afree[a], ((kc / kSlots) & 1) ^ 1, kSpinP);
      ok = __all_sync(0xffffffffu, ok && !*abort_flag);
      if (!ok) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        ct.abort = 1;
        break;
      }
      if (cid == 0) ct.consumed = kc + 1;
      tc::fence_after_sync();
      {
        // the box holds 32 rows a of 128 floats (l): this thread's column
        const float *wt =
            reinterpret_cast<const float *>(w_tile(s) + kh * G_HALF) + r;
        float h[32], lo[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const float v = wt[c * PT];
          h[c] = hi1(v);
          lo[c] = __fsub_rn(v, h[c]);
        }
        const uint32_t ta = aslots + lrow + 2 * PK * a + PH * kh;
        tc::tmem_st32(ta, h);
        tc::tmem_st32(ta + PK, lo);
      }
      tc::tmem_wait_st();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&ct.ready[a]);
    }
  }
  __syncwarp();

  pdl_trigger();
  if (warp >= 2 && warp < 6) {
    const bool ready =
        __all_sync(0xffffffffu, tc::mbar_wait(&ct.done, 0, kSpinP));
    if (!ready && lane == 0) atomicOr(err, kErrTimeout);
    const bool go = __all_sync(0xffffffffu, ready && !*abort_flag);
    if (go) {
      tc::fence_after_sync();
      const int q = warp & 3;
      const int l = l0 + q * 32 + lane;
      const uint32_t lrow = (uint32_t)(q * 32) << 16;
      float *out = FL + bm.fl_off + (int64_t)l * kp;
#pragma unroll 1
      for (int c0 = 0; c0 < B; c0 += 16) {
        if (c0 >= kp) break;                    // warp-uniform
        float v[16], w[16];
        acc_sum<B>(taddr + lrow, c0, v);
        acc_sum<B>(taddr + lrow, B + c0, w);
        if (l < bm.L) {
          // kp is a multiple of 4: whole float4s up to it
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const int j = c0 + 4 * c4;
            if (j < kp)
              *reinterpret_cast<float4 *>(out + j) =
                  make_float4(v[4 * c4] + w[4 * c4], v[4 * c4 + 1] + w[4 * c4 + 1],
                              v[4 * c4 + 2] + w[4 * c4 + 2],
                              v[4 * c4 + 3] + w[4 * c4 + 3]);
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && ct.abort) {
    for (int kc = ct.consumed; kc < ct.issued; ++kc)
      tc::mbar_wait(&ct.full[kc % S], (kc / S) & 1, kSpinP);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, kTmemCols);
}

// B form of F_s (s_pad x kp, row-major at fs_off) into the panel B-form
// layout at 2 x_off, columns kp .. B-1 zero: one CTA per 128-row tile.
template <int B>
__global__ void __launch_bounds__(128)
k_bform_fs(const BlockMeta *__restrict__ meta, const int2 *__restrict__ tiles,
           const float *__restrict__ Fs, int kp, float *__restrict__ out_bf) {
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  const BlockMeta bm = meta[t.x];
  const int r = t.y + threadIdx.x;
  if (r >= bm.s_pad) return;
  const float *src = Fs + bm.fs_off + (int64_t)r * kp;
  float *dst = out_bf + 2 * bm.x_off + (int64_t)(r >> 5) * 2 * B * 32 + (r & 31);
#pragma unroll 4
  for (int j = 0; j < B; ++j) {
    const float v = j < kp ? src[j] : 0.f;
    const float vh = hi1(v);
    dst[j * 32] = vh;
    dst[(B + j) * 32] = __fsub_rn(v, vh);
  }
}

// B form of a panel written by another kernel: one CTA per 128-row tile,
// one thread per row; the lanes of a warp write 32 consecutive positions of
// one chunk row.
template <int B>
__global__ void __launch_bounds__(128)
k_bform(const BlockMeta *__restrict__ meta, const SolverState *__restrict__ state,
        const int2 *__restrict__ tiles, const float *__restrict__ in,
        float *__restrict__ in_bf) {
  pdl_wait();
  pdl_trigger();
  const int2 t = tiles[blockIdx.x];
  if (state[t.x].status != kRunning) return;
  const BlockMeta bm = meta[t.x];
  const int r = t.y + threadIdx.x;
  if (r >= bm.s_pad) return;
  const float4 *src =
      reinterpret_cast<const float4 *>(in + bm.x_off + (int64_t)r * B);
  float *dst = in_bf + 2 * bm.x_off + (int64_t)(r >> 5) * 2 * B * 32 + (r & 31);
#pragma unroll
  for (int c4 = 0; c4 < B / 4; ++c4) {
    const float4 v = src[c4];
    const float4 vh = hi4(v), vl = sub4(v, vh);
    dst[(4 * c4 + 0) * 32] = vh.x;
    dst[(4 * c4 + 1) * 32] = vh.y;
    dst[(4 * c4 + 2) * 32] = vh.z;
    dst[(4 * c4 + 3) * 32] = vh.w;
    dst[(B + 4 * c4 + 0) * 32] = vl.x;
    dst[(B + 4 * c4 + 1) * 32] = vl.y;
    dst[(B + 4 * c4 + 2) * 32] = vl.z;
    dst[(B + 4 * c4 + 3) * 32] = vl.w;
  }
}

}  // namespace

cudaError_t launch_gpanel_tc(int32_t bsub, const BlockMeta *meta,
                             SolverState *state, const int2 *tiles,
                             int32_t ntiles, int32_t nctas, int32_t *ctl,
                             unsigned long long *ptime,
                             const CUtensorMap *gmaps,
                             const CUtensorMap *xmaps, const float *in,
                             const float *in2, float *out, float *out_bf,
                             int mode, int step, int32_t *err,
                             cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  nctas = nctas < ntiles ? nctas : ntiles;
  if (nctas < 1) nctas = 1;
  switch (bsub) {
    case 16: return launch_b<16>(meta, state, tiles, ntiles, nctas, ctl, ptime,
                                 gmaps, xmaps, in, in2, out, out_bf, mode, step,
                                 err, st);
    case 32: return launch_b<32>(meta, state, tiles, ntiles, nctas, ctl, ptime,
                                 gmaps, xmaps, in, in2, out, out_bf, mode, step,
                                 err, st);
    case 64: return launch_b<64>(meta, state, tiles, ntiles, nctas, ctl, ptime,
                                 gmaps, xmaps, in, in2, out, out_bf, mode, step,
                                 err, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_project_tc(int32_t bsub, const BlockMeta *meta,
                              const int2 *tiles, int32_t ntiles,
                              const CUtensorMap *wmaps,
                              const CUtensorMap *fmaps, float *FL, int32_t kp,
                              int32_t *err, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  auto go = [&](auto bw) -> cudaError_t {
    constexpr int B = decltype(bw)::value;
    static_assert(panel_tc_smem<B>() <= 227 * 1024, "shared memory");
    cudaError_t e = cudaFuncSetAttribute(
        k_project_tc<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)panel_tc_smem<B>());
    if (e != cudaSuccess) return e;
    return launch_pdl(k_project_tc<B>, dim3((unsigned)ntiles), dim3(kThreads),
                      panel_tc_smem<B>(), st, meta, tiles, wmaps, fmaps, FL,
                      (int)kp, err);
  };
  switch (bsub) {
    case 16: return go(std::integral_constant<int, 16>());
    case 32: return go(std::integral_constant<int, 32>());
    case 64: return go(std::integral_constant<int, 64>());
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_bform_fs(int32_t bsub, const BlockMeta *meta,
                            const int2 *tiles, int32_t ntiles, const float *Fs,
                            int32_t kp, float *out_bf, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (bsub) {
    case 16: return launch_pdl(k_bform_fs<16>, dim3(ntiles), dim3(128), 0, st,
                               meta, tiles, Fs, (int)kp, out_bf);
    case 32: return launch_pdl(k_bform_fs<32>, dim3(ntiles), dim3(128), 0, st,
                               meta, tiles, Fs, (int)kp, out_bf);
    case 64: return launch_pdl(k_bform_fs<64>, dim3(ntiles), dim3(128), 0, st,
                               meta, tiles, Fs, (int)kp, out_bf);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_bform(int32_t bsub, const BlockMeta *meta,
                         const SolverState *state, const int2 *tiles,
                         int32_t ntiles, const float *in, float *in_bf,
                         cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (bsub) {
    case 16: return launch_pdl(k_bform<16>, dim3(ntiles), dim3(128), 0, st, meta,
                               state, tiles, in, in_bf);
    case 32: return launch_pdl(k_bform<32>, dim3(ntiles), dim3(128), 0, st, meta,
                               state, tiles, in, in_bf);
    case 64: return launch_pdl(k_bform<64>, dim3(ntiles), dim3(128), 0, st, meta,
                               state, tiles, in, in_bf);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsvd
