// Split-precision tensor-core GEMM for sm_103a: tcgen05.mma with TMEM
// accumulators, operands staged in shared memory by TMA (cp.async.bulk.tensor).
//
//   C(m,n) = sum_k A[m][k] B[n][k]      A [M][lda], B [N][ldb] fp32, k contiguous
//
// This carries the two chi^2-class contractions of every Fig. 2(a) application
// (boundary x vectors, environment x vectors) and the tall-times-small products
// of the QR and truncation steps. FP32 inputs are split on chip into
// x = hi + lo, both rounded to TF32 (|x - hi - lo| <= 2^-22 |x|), and the
// product is a_lo b_hi + a_hi b_lo + a_hi b_hi (kind::tf32 MMAs, "3xTF32").
//
// The kernel is persistent (one CTA per SM, or one CTA pair per two SMs, walks a
// static tile schedule of 128x128, respectively 256x192, output tiles, optionally
// split over K). A's hi/lo tiles live in tensor
// memory: converter warps read one 128-byte row of the landed fp32 tile per
// thread and store hi and lo with tcgen05.st, so the MMAs take A from TMEM and
// only B's hi/lo tiles from shared memory.
//
// Shared memory bandwidth bounds the single-CTA form: per 32-term k-block an SM
// moves ~144 KB through it (TMA fills, the B split, the A rows, and 3 x 16 KB of B
// read by the MMAs), ~1150 cycles at 128 B/clock against 768 cycles of MMAs. When
// M spans more than one tile, CTA pairs (clusters of two, tcgen05 cta_group::2)
// compute 256x192 tiles instead: each CTA holds 128 rows of A in its TMEM and 96
// of the tile's 192 B rows in its shared memory, and rank 0 issues M=256, N=192
// MMAs that read B from both. Per output column, B's loads, split and MMA reads
// per SM halve. Converters and epilogue warps of both CTAs arrive on rank 0's
// barriers; MMA completion is signalled to both CTAs by a multicast commit. Each
// pair CTA has two sets of A converters taking alternate k-blocks.
//
// Accumulation: the tensor cores' FP32 accumulation over long K loses far more
// than round-to-nearest FP32 (measured ~1e-5 relative at K = 2048, ~1e-3 at
// K = 1e5). K is therefore cut into chunks of KCH_BLOCKS * BK = 256 terms; each
// chunk accumulates in a fresh TMEM accumulator and the epilogue warps add it to
// a running FP32 sum. A single CTA keeps that sum in TMEM (the MMAs of the next
// chunk wait for the drain; tiles of a single chunk alternate two accumulators
// instead, so a tile's MMAs overlap the previous tile's drain); a pair CTA keeps
// it in shared memory and always alternates two TMEM accumulators, so no chunk
// waits for a drain. Few output tiles are additionally split
// over K across CTAs, with the partials summed in FP64. Output blocks whose contiguous index is n
// pass through shared memory so that every store instruction is coalesced.
//
// Every wait on an mbarrier is bounded: a timeout sets an error word, the CTA
// stops issuing work, waits (bounded) for what it has in flight, frees its
// TMEM and exits; CTAs that start after an error return at once.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace fpeps {
namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = 32;   // BK fp32 = 128 bytes = one 128B swizzle row
constexpr int TILE_A = BM * BK * 4;   // bytes
constexpr int EPI_TILE = 32 * 33;                                 // floats: one warp's 32x32 output block
struct TcArgs {
  int64_t M, N, K;
  OutMap om;
  float* C;
  int* err;
  int m_fast;   // rasterisation: 1 => consecutive blocks walk m
  int64_t mt, nt;
  int ks;       // k-blocks per K slice (split-K); nsplit = ceil(nk / ks)
  int nsplit;
  int kch;      // k-blocks per TMEM accumulation chunk
  int nbuf;     // TMEM chunk accumulators: 2 (alternating) when every tile is one chunk or the
                // running sum is in shared memory (CTA pairs), else 1 (+ running sum in TMEM)
  int hold;     // self-test of the bounded waits: issue no loads, so every consumer times out
  float* part;  // nsplit > 1: partial results [nsplit][M][N] row-major
};

// Variant with the A operand in tensor memory. The converter warps of A read one
// 128-byte row of the landed fp32 tile each (one thread per TMEM lane), split it
// and store hi and lo straight into a TMEM slot with tcgen05.st; only B's hi/lo
// tiles stay in shared memory, so the MMAs read B alone from shared memory and the
// A split costs no shared-memory writes. TMEM columns of a single CTA: [0,128) a
// chunk accumulator; [128,256) a second one when every tile is a single chunk
// (chunks alternate, so the next chunk's MMAs overlap the drain), else the running
// FP32 sum; [256,512) four A slots of 32 hi + 32 lo columns, one per stage. A pair
// CTA: below. Warps: 0 TMA, 1 TMEM + MMA, 2..5 A converters (TMEM lane
// quarter = warp % 4), 6..7 and 12..15 B converters (in a pair CTA 12..15 are a
// second set of A converters), 8..11 epilogue, 16 barrier waiter for the MMA warp,
// 17..18 two more B converters (pair CTA; idle in a single CTA).
constexpr int P_THREADS = 608;
// Pair tiles are 256 x 192 (N = 192 per MMA): a tcgen05.mma costs its issuing thread a
// fixed ~58 ns (~120 SM cycles at 2.07 GHz, measured on GB300, M = 128 per SM, kind::tf32)
// for any N up to ~200, while an N = 128 pair MMA gives each SM only ~70 cycles of tensor
// work; N = 192 does 1.5x the work per MMA at the same cost. TMEM of a pair CTA: two
// 192-column accumulators [0,384) and two A slots [384,512) (an A-slot ring of its own,
// freed by the MMAs of the k-block two back); shared memory: three 40 KB stages and the
// running sum, which also stages the final output tile (no separate epilogue tiles).
template <bool PAIR> __host__ __device__ constexpr int t_bn() { return PAIR ? 192 : BN; }   // output columns per tile
template <bool PAIR> __host__ __device__ constexpr int t_stages() { return PAIR ? 3 : 4; }
template <bool PAIR> __host__ __device__ constexpr int t_aslots() { return PAIR ? 2 : 4; }
template <bool PAIR> __host__ __device__ constexpr uint32_t t_aslot_base() { return PAIR ? 2 * 192 : 2 * BN; }
// Shared memory: the stage ring (A fp32 | B hi (in place) | B lo; a pair CTA holds
// half of the tile's B rows), then in a pair CTA the running FP32 sum of multi-chunk
// tiles (128 rows x (BN + 1) floats, padded so that a row per lane is conflict-free),
// the barriers, and in a single CTA the epilogue's 32x33 tiles.
template <bool PAIR> __host__ __device__ constexpr int t_stage_bytes() {
  return TILE_A + 2 * (t_bn<PAIR>() / (PAIR ? 2 : 1)) * BK * 4;
}
template <bool PAIR> __host__ __device__ constexpr int t_run_bytes() { return PAIR ? BM * (t_bn<PAIR>() + 1) * 4 : 0; }
template <bool PAIR> __host__ __device__ constexpr int t_bar_off() { return t_stages<PAIR>() * t_stage_bytes<PAIR>() + t_run_bytes<PAIR>(); }
template <bool PAIR> __host__ __device__ constexpr int t_smem_bytes() {
  return t_bar_off<PAIR>() + 256 + (PAIR ? 0 : 4 * EPI_TILE * 4) + 1024;
}
static_assert(t_smem_bytes<false>() <= 227 * 1024 && t_smem_bytes<true>() <= 227 * 1024, "shared memory");
static_assert(2 * t_bn<true>() + 2 * 64 <= 512 && 2 * BN + 4 * 64 <= 512, "tensor memory");
constexpr uint32_t T_RUN = BN;   // single CTA: TMEM column base of the running sum (see the layout above)
// warps: 0 TMA, 1 TMEM + MMA, 2..5 A converters, 6..7 and 12..15 B converters, 8..11 epilogue,
// 16 waiter, 17..18 B converters (pair); in a pair CTA 12..15 are a second set of A converters
constexpr int T_BCONV0 = 6, T_NBCONV = 6, T_EPI0 = 8, T_BCONV1 = 12, T_WAITER = 16, T_BCONV2 = 17;

// named barrier 1 between the MMA warp and the waiter warp (64 threads); returns
// true if any participating thread passed true
__device__ __forceinline__ bool handoff_abort(bool mine) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 64, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)mine)
      : "memory");
  return r != 0;
}

// BF: the BF16x3 form (kind::f16 MMAs with BF16 hi/lo splits, K = 16 per MMA): A's hi/lo slots
// are half as wide (two BF16 per TMEM column), B's BF16 hi/lo go to a no-swizzle K-major image
// beside the landed FP32 tile, and a k-block takes 6 MMAs instead of 12.
template <bool PAIR, bool BF>
__global__ void __launch_bounds__(P_THREADS, 1) k_gemm_tf32x3_t(const __grid_constant__ CUtensorMap mapA,
                                                                const __grid_constant__ CUtensorMap mapB, TcArgs g) {
  // CTA pair (cluster of two): each CTA holds 128 rows of a 256-row tile (A in its
  // TMEM, accumulator in its TMEM) and half of the tile's B columns in its shared
  // memory; rank 0 issues the M=256 MMAs for both.
  constexpr int CS = PAIR ? 2 : 1;
  constexpr int BNT = t_bn<PAIR>();            // output columns per tile
  constexpr int BNH = BNT / CS;                // B rows (output columns) held by this CTA
  constexpr int TILE_BH = BNH * BK * 4;        // bytes
  constexpr int T_STAGE_BYTES = t_stage_bytes<PAIR>();
  constexpr int T_STAGES = t_stages<PAIR>();
  constexpr int NSLOT = t_aslots<PAIR>();      // A slots in TMEM (single CTA: one per stage)
  // A converter sets: each converts every NAS-th k-block, so a warp has NAS k-block
  // periods for its load/split/TMEM-store chain. In a pair CTA warps 12..15 are the
  // second set and B, halved per CTA, is converted by warps 6..7 and 17..18.
  constexpr int NAS = PAIR ? 2 : 1;
  constexpr int NBW = PAIR ? 4 : T_NBCONV;
  const uint32_t rank = PAIR ? cluster_rank() : 0;
  const bool issuer = rank == 0;
  // a CTA pair may not split up on a shared early exit, so only single CTAs return here
  if (!PAIR && *(volatile int*)g.err) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + t_bar_off<PAIR>());
  uint64_t* bconv = full + T_STAGES;
  uint64_t* empty = bconv + T_STAGES;
  uint64_t* aconv = empty + T_STAGES;   // [4] A slot filled
  uint64_t* aempty = aconv + 4;         // [2] pair CTA: A slot free (MMAs of its last k-block done)
  uint64_t* accf = aempty + 2;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  float* epi_tiles = (float*)(smem + t_bar_off<PAIR>() + 256);
  float* run_sum = (float*)(smem + T_STAGES * T_STAGE_BYTES);   // pair CTA: [BM][BNT + 1]

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t ntiles = g.mt * g.nt * g.nsplit;
  const int64_t tile0 = blockIdx.x / CS, tstep = gridDim.x / CS;
  const int nk_all = (int)((g.K + BK - 1) / BK);
  auto kslice = [&](int64_t tile, int& kb0, int& nk) {
    const int split = (int)(tile / (g.mt * g.nt));
    kb0 = split * g.ks;
    nk = min(g.ks, nk_all - kb0);
  };
  auto A_f = [&](int st) { return smem + st * T_STAGE_BYTES; };
  auto B_hi = [&](int st) { return smem + st * T_STAGE_BYTES + TILE_A; };
  auto B_lo = [&](int st) { return smem + st * T_STAGE_BYTES + TILE_A + TILE_BH; };
  // BF16 images of B (BF): hi then lo, element (n, k) at (k / 8) LB + (n / 8) 128 + (n % 8) 16 + (k % 8) 2
  constexpr uint32_t LB = (uint32_t)(BNH / 8) * 128;   // K-direction core-matrix stride of a BF16 image
  auto B_h16 = [&](int st) { return smem + st * T_STAGE_BYTES + TILE_A + TILE_BH; };
  auto B_l16 = [&](int st) { return smem + st * T_STAGE_BYTES + TILE_A + TILE_BH + TILE_BH / 2; };
  constexpr uint32_t AW = BF ? 32 : 64;                 // TMEM columns of an A slot (hi, then lo)
  auto tile_mn = [&](int64_t tile, int64_t& m0, int64_t& n0) {
    tile %= g.mt * g.nt;
    const int64_t mt = g.m_fast ? tile % g.mt : tile / g.nt;
    const int64_t nt = g.m_fast ? tile / g.mt : tile % g.nt;
    m0 = mt * (BM * CS) + rank * BM;
    n0 = nt * BNT;
  };

  if (threadIdx.x == 0) {
    for (int st = 0; st < T_STAGES; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&bconv[st], NBW * CS);
      mbar_init(&empty[st], 1);
    }
    for (int b = 0; b < 4; ++b) mbar_init(&aconv[b], 4 * CS);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&aempty[b], 1);
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4 * CS);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (PAIR) {   // one warp of each CTA of the pair, collectively
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(4 * BN));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(4 * BN));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if constexpr (PAIR) cluster_sync_all();   // the peer's barriers are initialised before any remote arrival
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // A slots: 64 columns each (32 hi + 32 lo) from column abase
  const uint32_t abase = t_aslot_base<PAIR>();

  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
      int it = 0;
      bool ok = !g.hold;
      for (int64_t tile = tile0; tile < ntiles && ok; tile += tstep) {
        int64_t m0, n0;
        tile_mn(tile, m0, n0);
        int kb0, nk;
        kslice(tile, kb0, nk);
        for (int kb = 0; kb < nk; ++kb, ++it) {
          const int st = it % T_STAGES;
          if (!mbar_wait(&empty[st], ((it / T_STAGES) & 1) ^ 1, abort_flag)) { ok = false; break; }
          mbar_arrive_expect_tx(&full[st], TILE_A + TILE_BH);
          tma_load_2d(A_f(st), &mapA, &full[st], (kb0 + kb) * BK, (int)m0);
          tma_load_2d(B_hi(st), &mapB, &full[st], (kb0 + kb) * BK, (int)(n0 + rank * BNH));
          ++issued;
        }
      }
    }
  } else if (warp == 1 && issuer) {
    // The MMA warp touches no shared memory while MMAs are in flight: an mbarrier
    // wait by the thread that issued tcgen05.mma stalls it until those MMAs have
    // drained (measured: one wait per 12 MMAs halves the tensor-pipe rate). The
    // waiter warp does the mbarrier waits and hands each ready k-block over on a
    // named barrier, whose OR-reduction also carries an abort.
    // D FP32; A, B TF32 (2) or BF16 (1); N; M
    const uint32_t idesc = (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) |
                           ((uint32_t)(BNT >> 3) << 17) | ((uint32_t)((BM * CS) >> 4) << 24);
    int it = 0, lc = 0;
    bool ok = true;
    for (int64_t tile = tile0; tile < ntiles && ok; tile += tstep) {
      int kb0, nk;
      kslice(tile, kb0, nk);
      for (int c0 = 0; c0 < nk && ok; c0 += g.kch, ++lc) {
        const int buf = lc % g.nbuf;
        const uint32_t d = tmem + (uint32_t)(buf * BNT);
        const int c1 = min(nk, c0 + g.kch);
        for (int kb = c0; kb < c1; ++kb, ++it) {
          if (handoff_abort(false)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int st = it % T_STAGES, as = PAIR ? it % NSLOT : st;
          if (lane == 0) {
            const uint32_t ah = tmem + abase + (uint32_t)(as * AW), al = ah + AW / 2;
            if constexpr (BF) {
              const uint8_t* bh = B_h16(st);
              const uint8_t* bl = B_l16(st);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {   // K = 16 per MMA: two core-matrix columns
                const uint64_t dh = sdesc_noswz(bh + 2 * kk * LB, LB, 128), dl = sdesc_noswz(bl + 2 * kk * LB, LB, 128);
                mma_bf16_ts<PAIR>(d, al + (uint32_t)(kk * 8), dh, idesc, ((kb - c0) | kk) ? 1u : 0u);
                mma_bf16_ts<PAIR>(d, ah + (uint32_t)(kk * 8), dl, idesc, 1u);
                mma_bf16_ts<PAIR>(d, ah + (uint32_t)(kk * 8), dh, idesc, 1u);
              }
            } else {
              const uint64_t bh = sdesc(B_hi(st)), bl = sdesc(B_lo(st));
#pragma unroll
              for (int kk = 0; kk < BK / 8; ++kk) {
                const uint64_t o = (uint64_t)(kk * 32) >> 4;
                mma_tf32_ts<PAIR>(d, al + (uint32_t)(kk * 8), bh + o, idesc, ((kb - c0) | kk) ? 1u : 0u);
                mma_tf32_ts<PAIR>(d, ah + (uint32_t)(kk * 8), bl + o, idesc, 1u);
                mma_tf32_ts<PAIR>(d, ah + (uint32_t)(kk * 8), bh + o, idesc, 1u);
              }
            }
            mma_commit<PAIR>(&empty[st], (1u << CS) - 1);   // frees the stage (both CTAs) ...
            if constexpr (PAIR) mma_commit<PAIR>(&aempty[as], (1u << CS) - 1);   // ... and the A slot
            if (kb + 1 == c1) mma_commit<PAIR>(&accf[buf], (1u << CS) - 1);
          }
          __syncwarp();
        }
      }
    }
    if (lane == 0) {
      mma_commit<PAIR>(drain, 1);
      const unsigned long long t0 = clock64();
      while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_LIMIT) {
      }
    }
    __syncwarp();
  } else if (warp == T_WAITER && issuer) {
    // waits for the inputs of every k-block (and, at a chunk start, for the
    // accumulator buffer) in the MMA warp's order, then hands the k-block over
    int it = 0, lc = 0;
    bool ok = true;
    for (int64_t tile = tile0; tile < ntiles && ok; tile += tstep) {
      int kb0, nk;
      kslice(tile, kb0, nk);
      for (int c0 = 0; c0 < nk && ok; c0 += g.kch, ++lc) {
        const int buf = lc % g.nbuf;
        const int c1 = min(nk, c0 + g.kch);
        for (int kb = c0; kb < c1; ++kb, ++it) {
          const int st = it % T_STAGES, as = PAIR ? it % NSLOT : st;
          bool ready = true;
          if (kb == c0) ready = mbar_wait(&acce[buf], ((lc / g.nbuf) & 1) ^ 1, abort_flag);
          ready = ready && mbar_wait(&bconv[st], (it / T_STAGES) & 1, abort_flag);
          ready = ready && mbar_wait(&aconv[as], (it / NSLOT) & 1, abort_flag);
          // relay the converters' tensor-memory stores to the MMA warp
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          const bool any_abort = handoff_abort(!__all_sync(0xffffffffu, ready));
          if (any_abort) { ok = false; break; }
        }
      }
    }
  } else if ((warp >= 2 && warp < T_BCONV0) || (PAIR && warp >= T_BCONV1 && warp < T_WAITER)) {
    // A converters: thread = TMEM lane = tile row
    const int quarter = warp % 4;
    const int set = warp >= T_BCONV1 ? 1 : 0;
    const int r = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    int it = 0;
    bool ok = true;
    for (int64_t tile = tile0; tile < ntiles && ok; tile += tstep) {
      int kb0, nk;
      kslice(tile, kb0, nk);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        if (NAS > 1 && it % NAS != set) continue;
        const int st = it % T_STAGES, as = PAIR ? it % NSLOT : st;
        // the slot is free once the MMAs of its previous k-block are done. Single CTA: the
        // slot is the stage's, and the TMA refill of the stage waited for the same release,
        // so this wait passes at once; pair CTA: the A-slot ring of its own (two back).
        // In a pair CTA a converter set sees a stage only every other fill when the ring
        // length is odd, so a parity wait on full[st] alone could match the fill two back
        // while the previous one is still landing. The slot wait comes first: once the MMAs
        // of k-block it - 2 are done, the fill of it - T_STAGES has landed (those MMAs
        // consumed it), so full[st] is in the phase of k-block it and the parity is exact.
        if (PAIR ? !mbar_wait(&aempty[as], ((it / NSLOT) & 1) ^ 1, abort_flag)
                 : !mbar_wait(&empty[st], ((it / T_STAGES) & 1) ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        if (!mbar_wait(&full[st], (it / T_STAGES) & 1, abort_flag)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint4* row = (const uint4*)(A_f(st) + r * 128);
        if constexpr (BF) {
          // two BF16 per TMEM column (the lower K index in the lower half)
          uint32_t h2[16], l2[16];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint4 v = row[c ^ (r & 7)];   // 128-byte swizzle: chunk c of row r
            uint32_t h[4], l[4];
            bf16_split(__uint_as_float(v.x), h[0], l[0]);
            bf16_split(__uint_as_float(v.y), h[1], l[1]);
            bf16_split(__uint_as_float(v.z), h[2], l[2]);
            bf16_split(__uint_as_float(v.w), h[3], l[3]);
            h2[2 * c] = bf16_pack(h[0], h[1]);
            h2[2 * c + 1] = bf16_pack(h[2], h[3]);
            l2[2 * c] = bf16_pack(l[0], l[1]);
            l2[2 * c + 1] = bf16_pack(l[2], l[3]);
          }
          const uint32_t ta = tmem + lane_base + abase + (uint32_t)(as * AW);
          tmem_st16(ta, h2);
          tmem_st16(ta + AW / 2, l2);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive_issuer<PAIR>(&aconv[as], rank);
          continue;
        }
        float hi[32], lo[32];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint4 v = row[c ^ (r & 7)];   // 128-byte swizzle: chunk c of row r
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint32_t h = tf32_round(w[e]);
            hi[c * 4 + e] = __uint_as_float(h);
            lo[c * 4 + e] = __uint_as_float(tf32_round(__float_as_uint(__uint_as_float(w[e]) - __uint_as_float(h))));
          }
        }
        const uint32_t ta = tmem + lane_base + abase + (uint32_t)(as * AW);
        tmem_st32(ta, hi);
        tmem_st32(ta + 32, lo);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_issuer<PAIR>(&aconv[as], rank);
      }
    }
  } else if ((warp >= T_BCONV0 && warp < T_EPI0) || (!PAIR && warp >= T_BCONV1 && warp < T_WAITER) ||
             (PAIR && warp >= T_BCONV2 && warp < T_BCONV2 + 2)) {
    // B converters: hi in place, lo into the second B tile
    const int cw = warp < T_EPI0 ? warp - T_BCONV0
                                 : (PAIR ? warp - T_BCONV2 : warp - T_BCONV1) + (T_EPI0 - T_BCONV0);
    int it = 0;
    bool ok = true;
    for (int64_t tile = tile0; tile < ntiles && ok; tile += tstep) {
      int kb0, nk;
      kslice(tile, kb0, nk);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int st = it % T_STAGES;
        if (!mbar_wait(&full[st], (it / T_STAGES) & 1, abort_flag)) { ok = false; break; }
        if constexpr (BF) {
          // the landed FP32 tile (128-byte swizzle) -> BF16 hi and lo images, 4 elements per step
          const uint4* src = (const uint4*)B_hi(st);
          uint8_t* h16 = B_h16(st);
          uint8_t* l16 = B_l16(st);
          for (int e = cw * 32 + lane; e < TILE_BH / 32; e += NBW * 32) {
            // row n, 8-element group j (k = 8j .. 8j+7). Lanes walk rows: a quarter warp reads eight
            // distinct 16-byte columns of the swizzled tile and writes 128 contiguous bytes
            const int n = e % BNH, j = e / BNH;
            const uint4 v0 = src[n * 8 + ((2 * j) ^ (n & 7))];
            const uint4 v1 = src[n * 8 + ((2 * j + 1) ^ (n & 7))];
            const float f[8] = {__uint_as_float(v0.x), __uint_as_float(v0.y), __uint_as_float(v0.z),
                                __uint_as_float(v0.w), __uint_as_float(v1.x), __uint_as_float(v1.y),
                                __uint_as_float(v1.z), __uint_as_float(v1.w)};
            uint32_t h[8], l[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) bf16_split(f[q], h[q], l[q]);
            const uint32_t off = (uint32_t)j * LB + (uint32_t)(n / 8) * 128 + (uint32_t)(n % 8) * 16;
            *(uint4*)(h16 + off) = make_uint4(bf16_pack(h[0], h[1]), bf16_pack(h[2], h[3]),
                                              bf16_pack(h[4], h[5]), bf16_pack(h[6], h[7]));
            *(uint4*)(l16 + off) = make_uint4(bf16_pack(l[0], l[1]), bf16_pack(l[2], l[3]),
                                              bf16_pack(l[4], l[5]), bf16_pack(l[6], l[7]));
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive_issuer<PAIR>(&bconv[st], rank);
          continue;
        }
        uint4* bh = (uint4*)B_hi(st);
        uint4* blo = (uint4*)B_lo(st);
#pragma unroll 3
        for (int e = cw * 32 + lane; e < TILE_BH / 16; e += NBW * 32) {
          const uint4 v = bh[e];
          const uint4 h = make_uint4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
          const uint4 l = make_uint4(tf32_round(__float_as_uint(__uint_as_float(v.x) - __uint_as_float(h.x))),
                                     tf32_round(__float_as_uint(__uint_as_float(v.y) - __uint_as_float(h.y))),
                                     tf32_round(__float_as_uint(__uint_as_float(v.z) - __uint_as_float(h.z))),
                                     tf32_round(__float_as_uint(__uint_as_float(v.w) - __uint_as_float(h.w))));
          bh[e] = h;
          blo[e] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_issuer<PAIR>(&bconv[st], rank);
      }
    }
  } else if (warp >= T_EPI0 && warp < T_BCONV1) {
    const int q = warp - T_EPI0;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    int lc = 0;
    bool ok = true;
    for (int64_t tile = tile0; tile < ntiles && ok; tile += tstep) {
      int64_t m0, n0;
      tile_mn(tile, m0, n0);
      int kb0, nk;
      kslice(tile, kb0, nk);
      const int nch = (nk + g.kch - 1) / g.kch;
      const int64_t m = m0 + q * 32 + lane;
      const bool mrow = m < g.M;
      const int64_t mo = mrow ? (m / g.om.mdiv) * g.om.c0 + (m % g.om.mdiv) * g.om.c1 : 0;
      for (int ch = 0; ch < nch; ++ch, ++lc) {
        const int buf = lc % g.nbuf;
        if (!mbar_wait(&accf[buf], (lc / g.nbuf) & 1, abort_flag)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
        for (int cb = 0; cb < BNT; cb += 32) {
          float v[32];
          uint32_t rc[32], rr[32];
          tmem_ld32_async(tmem + lane_base + (uint32_t)(buf * BNT + cb), rc);
          if (ch == 0) {
            tmem_wait32(rc);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(rc[j]);
          } else if constexpr (PAIR) {
            const float* rs = run_sum + (q * 32 + lane) * (BNT + 1) + cb;
            tmem_wait32(rc);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = rs[j] + __uint_as_float(rc[j]);
          } else {
            tmem_ld32_async(tmem + lane_base + T_RUN + (uint32_t)cb, rr);
            tmem_wait32(rc);
            tmem_wait32(rr);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(rr[j]) + __uint_as_float(rc[j]);
          }
          if (ch + 1 < nch) {
            if constexpr (PAIR) {
              float* rs = run_sum + (q * 32 + lane) * (BNT + 1) + cb;
#pragma unroll
              for (int j = 0; j < 32; ++j) rs[j] = v[j];
            } else {
              tmem_st32(tmem + lane_base + T_RUN + (uint32_t)cb, v);
            }
          } else if (!__shfl_sync(0xffffffffu, *abort_flag, 0)) {   // warp-uniform decision
            if (g.nsplit > 1 || g.om.c3 == 1) {
              // staging of this warp's 32 x 32 block: its own rows of the running sum in a pair
              // CTA (the tile's last use of them), else the warp's epilogue tile
              constexpr int TS = PAIR ? BNT + 1 : 33;
              float* tw = PAIR ? run_sum + (q * 32) * TS + cb : epi_tiles + q * EPI_TILE;
#pragma unroll
              for (int j = 0; j < 32; ++j) tw[lane * TS + j] = v[j];
              __syncwarp();
              const int64_t n = n0 + cb + lane;
              const bool ncol = n < g.N;
              if (g.nsplit > 1) {
                float* pbase = g.part + (tile / (g.mt * g.nt)) * g.M * g.N + n;
                for (int r = 0; r < 32; ++r) {
                  const int64_t mr = m0 + q * 32 + r;
                  if (mr < g.M && ncol) pbase[mr * g.N] = tw[r * TS + lane];
                }
              } else {
                const int64_t no = ncol ? (n / g.om.ndiv) * g.om.c2 + (n % g.om.ndiv) : 0;
                for (int r = 0; r < 32; ++r) {
                  const int64_t mor = __shfl_sync(0xffffffffu, mo, r);
                  const int64_t mr = m0 + q * 32 + r;
                  if (mr < g.M && ncol) g.C[mor + no] = tw[r * TS + lane];
                }
              }
              __syncwarp();
            } else if (mrow) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const int64_t n = n0 + cb + j;
                if (n < g.N) g.C[mo + (n / g.om.ndiv) * g.om.c2 + (n % g.om.ndiv) * g.om.c3] = v[j];
              }
            }
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_issuer<PAIR>(&acce[buf], rank);
      }
    }
  }

  // every role has left its loop (finished or aborted) once all threads meet here;
  // only then is the abort flag final
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag) {
    if (warp == 0 && lane == 0) {   // wait (bounded) for the TMA loads still in flight
      for (int it = issued > T_STAGES ? issued - T_STAGES : 0; it < issued; ++it) {
        const int st = it % T_STAGES;
        const unsigned long long t0 = clock64();
        while (!mbar_try_wait(&full[st], (it / T_STAGES) & 1) && clock64() - t0 < WAIT_LIMIT) {
        }
      }
    }
    if (threadIdx.x == 0) atomicExch(g.err, 1);
  }
  __syncthreads();
  // the pair's MMAs read this CTA's shared memory and write its TMEM, and the peer
  // arrives on this CTA's barriers: neither CTA frees or exits before both are here
  if constexpr (PAIR) cluster_sync_all();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if constexpr (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * BN));
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * BN));
  }
}

// Sum of the K-slice partials in FP64, written through the output map.
__global__ void k_splitk_reduce(const float* __restrict__ part, int nsplit, int64_t M, int64_t N, OutMap om,
                                float* __restrict__ C) {
  const int64_t tot = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) acc += (double)part[sp * tot + e];
    const int64_t m = e / N, n = e % N;
    C[(m / om.mdiv) * om.c0 + (m % om.mdiv) * om.c1 + (n / om.ndiv) * om.c2 + (n % om.ndiv) * om.c3] = (float)acc;
  }
}

// ---------------------------------------------------------------- host side
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  });
  FP_CHECK(fn != nullptr, FPEPS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  return fn;
}

CUtensorMap make_map(const float* base, int64_t rows, int64_t K, int64_t ld, int box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  FP_CHECK(r == CUDA_SUCCESS, FPEPS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

bool gemm_tc_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb) {
  // TMA: 16-byte aligned row strides, at least one full k-box; rows of a box that
  // fall outside M or N are filled with zeros and never stored
  return M >= 1 && N >= 1 && K >= BK && (lda % 4) == 0 && (ldb % 4) == 0 && lda >= K && ldb >= K &&
         M < (1LL << 31) && N < (1LL << 31) && K < (1LL << 31);
}

constexpr int KCH_BLOCKS = 8;   // 256 terms per TMEM accumulation chunk (K <= 512: one chunk)

// split over K only to fill the SMs when there are few output tiles
static int nsplit_of(int64_t tiles, int64_t K, int sms) {
  const int64_t nk = (K + BK - 1) / BK;
  int best = 1;
  double best_eff = 0;
  for (int sp = 1; sp <= 64; ++sp) {
    if ((int64_t)sp * KCH_BLOCKS > nk) break;
    const int64_t t = tiles * sp;
    const double eff = (double)t / (double)(((t + sms - 1) / sms) * sms);
    if (eff > best_eff + 0.02) { best = sp; best_eff = eff; }
    if (eff >= 0.9) break;
  }
  return best;
}

static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    FP_CUDA(cudaGetDevice(&dev));
    FP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

// CTA pairs the GPU holds at once (clusters of two CTAs, one CTA per SM); 0 if
// the pair kernel cannot be launched
static int pair_slots() {
  static int n = -1;
  if (n < 0) {
    FP_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3_t<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 t_smem_bytes<true>()));
    FP_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3_t<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 t_smem_bytes<true>()));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sm_count() & ~1));
    cfg.blockDim = dim3(P_THREADS);
    cfg.dynamicSmemBytes = t_smem_bytes<true>();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, k_gemm_tf32x3_t<true, false>, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      c = 0;
    }
    n = c;
  }
  return n;
}

// Tile schedule of one product: CTA pairs (256-row tiles) whenever M spans more
// than one 128-row tile, single CTAs otherwise; K split only to fill the GPU.
struct Plan {
  bool pair;
  int64_t mt, nt, slots;
  int ks, nsplit;
};
static Plan plan_of(int64_t M, int64_t N, int64_t K) {
  Plan p;
  p.pair = M > BM && pair_slots() > 0;
  const int cs = p.pair ? 2 : 1;
  p.slots = p.pair ? pair_slots() : sm_count();
  p.mt = (M + BM * cs - 1) / (BM * cs);
  p.nt = (N + (p.pair ? t_bn<true>() : BN) - 1) / (p.pair ? t_bn<true>() : BN);
  const int64_t nk = (K + BK - 1) / BK;
  const int ns = nsplit_of(p.mt * p.nt, K, (int)p.slots);
  p.ks = (int)((nk + ns - 1) / ns);
  p.nsplit = (int)((nk + p.ks - 1) / p.ks);   // every slice non-empty
  return p;
}

size_t gemm_tc_scratch_bytes(int, int64_t M, int64_t N, int64_t K) {
  const Plan p = plan_of(M, N, K);
  return 256 + (p.nsplit > 1 ? (size_t)p.nsplit * M * N * sizeof(float) : 0);
}

void gemm_tc(cudaStream_t s, int mode, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
             int64_t ldb, float* C, OutMap om, void* scratch, size_t scratch_bytes, bool hold_loads) {
  FP_CHECK(mode == FPEPS_TF32X3 || mode == FPEPS_BF16X3, FPEPS_ERR_UNSUPPORTED, "tensor-core GEMM: 3xTF32 or 3xBF16");
  const bool bf = mode == FPEPS_BF16X3;
  FP_CHECK(scratch && scratch_bytes >= sizeof(int), FPEPS_ERR_ARG, "tensor-core GEMM: scratch");
  FP_CHECK(((uintptr_t)A % 16) == 0 && ((uintptr_t)B % 16) == 0, FPEPS_ERR_ARG, "tensor-core GEMM: operand alignment");
  static bool attr = false;
  if (!attr) {
    FP_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3_t<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 t_smem_bytes<false>()));
    FP_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3_t<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 t_smem_bytes<false>()));
    attr = true;
  }
  const Plan p = plan_of(M, N, K);
  CUtensorMap ma = make_map(A, M, K, lda, BM);
  CUtensorMap mb = make_map(B, N, K, ldb, p.pair ? t_bn<true>() / 2 : BN);
  TcArgs g;
  g.M = M; g.N = N; g.K = K; g.om = om; g.C = C; g.err = (int*)scratch;
  g.mt = p.mt;
  g.nt = p.nt;
  g.m_fast = g.mt <= g.nt ? 1 : 0;
  g.ks = p.ks;
  g.nsplit = p.nsplit;
  g.kch = g.ks <= 2 * KCH_BLOCKS ? g.ks : KCH_BLOCKS;
  g.nbuf = (p.pair || (g.ks + g.kch - 1) / g.kch == 1) ? 2 : 1;
  g.hold = hold_loads ? 1 : 0;
  g.part = nullptr;
  if (g.nsplit > 1) {
    FP_CHECK(scratch_bytes >= gemm_tc_scratch_bytes(mode, M, N, K), FPEPS_ERR_ARG, "tensor-core GEMM: scratch too small");
    g.part = (float*)((char*)scratch + 256);
  }
  const int64_t tiles = g.mt * g.nt * g.nsplit;
  FP_CHECK(tiles < (1LL << 30), FPEPS_ERR_UNSUPPORTED, "tensor-core GEMM: grid too large");
  ProfToken pt = prof_begin(PROF_GEMM_TC, s, 2.0 * M * N * K, 4.0 * ((double)M * K + (double)N * K + (double)M * N));
  if (p.pair) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * std::min<int64_t>(tiles, p.slots)));
    cfg.blockDim = dim3(P_THREADS);
    cfg.dynamicSmemBytes = t_smem_bytes<true>();
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (bf) FP_CUDA(cudaLaunchKernelEx(&cfg, k_gemm_tf32x3_t<true, true>, ma, mb, g));
    else FP_CUDA(cudaLaunchKernelEx(&cfg, k_gemm_tf32x3_t<true, false>, ma, mb, g));
  } else {
    const unsigned grid1 = (unsigned)std::min<int64_t>(tiles, p.slots);
    if (bf) k_gemm_tf32x3_t<false, true><<<grid1, P_THREADS, t_smem_bytes<false>(), s>>>(ma, mb, g);
    else k_gemm_tf32x3_t<false, false><<<grid1, P_THREADS, t_smem_bytes<false>(), s>>>(ma, mb, g);
  }
  FP_LAUNCH();
  if (g.nsplit > 1) {
    const int64_t tot = M * N;
    const int rb = (int)std::min<int64_t>((tot + 255) / 256, 152 * 16);
    k_splitk_reduce<<<rb, 256, 0, s>>>(g.part, g.nsplit, M, N, om, C);
    FP_LAUNCH();
  }
  prof_end(pt, s);
}

}  // namespace fpeps
