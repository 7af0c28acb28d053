// The site sandwich on the tcgen05 tensor cores (3xTF32, sm_103a).
//
// Same operation as sandwich.cu (Sec. III: the sandwich of ket, PEPO and bra is
// applied to blocks of vectors with the PEPO indices kept separate): for every
// block I[X][Y] of the input, X = (x, x_w, x'), Y = (y, y_w, y'), and every output
// pair (v_w, z_w) with at least one PEPO channel,
//   ket  D1[(b,x',y'), (q,v,z)] = sum_{ch of the pair} sum_{(x,y)} I_ch[(b,x',y'),(x,y)] AW_ch[(x,y),(q,v,z)]
//   bra  D2[(b,v,z), (v',z')]  = sum_q sum_{(x',y')} D1[(b,x',y'),(q,v,z)] A[(x',y'),q,(v',z')]
//   O[(v,v_w,v'),(z,z_w,z')] = D2
// where I_ch is I restricted to the channel's (x_w, y_w) and AW_ch = A . W_ch.
//
// Both steps are 128-row tcgen05 MMAs (kind::tf32, FP32 accumulators in tensor
// memory), with every operand split x = hi + lo (TF32) and the product
// lo*hi + hi*lo + hi*hi. A group of nb consecutive blocks fills the 128 rows.
//   * ket A (the gathered input rows) is split by producer warps straight into
//     tensor memory; ket B (AW_ch, a per-site constant) is pre-split into hi/lo
//     images in the MMA's K-major layout and fetched per channel by bulk copies.
//   * D1 is moved by a transposer warpgroup through shared memory into the bra's
//     A operand (rows (b,v,z), K = (x',y')), one physical index q at a time into
//     two alternating tensor-memory slots; the bra B images (per q) stay
//     resident in shared memory.
//   * D2 leaves through shared memory with coalesced stores: the output bundle of
//     unit stride is stored PEPO-index outermost (bundle_index), so every output pair
//     owns contiguous runs.
// Warp roles (16 warps): 0 bulk copies, 1 tensor-memory allocation and the ket MMAs, 2-3 the
// bra MMAs (one warp per bra-A slot, each into its own half of D2), 4-7 ket-A producers, 8-11
// epilogue (adds the D2 halves; releases D2 before its stores), 12-15 transposer. A tcgen05.mma
// occupies its issuing thread for roughly the same ~100 cycles at any N up to ~200 (measured on
// GB300, M = 128, kind::tf32), so the narrow bra products are issued from two threads, and the ket
// of the next pair, issued from a third, overlaps the bra of the current one. Every wait is
// bounded; on a timeout the CTA raises its abort flag, waits (bounded) for its bulk copies and
// MMAs, frees its tensor memory and exits.
#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace fpeps {
namespace {

using namespace tc;

constexpr int SW_THREADS = 512;
constexpr int KPAD = 40;            // padded K (multiple of 8) of both steps: (x,y) and (x',y') <= 36 terms
constexpr int N1MAX = 144;          // ket N: (q, v, z)
constexpr int N2MAX = 48;           // bra N: (v', z') <= 36, padded to 16
constexpr int PMAX = 4;             // physical dimension
constexpr int RMAX = 36;            // rows per block of either step
constexpr int KB_STAGES = 2;
constexpr uint32_t KB_IMG = N1MAX * KPAD * 4;   // bytes of one ket-B image (hi or lo) at the largest shape
constexpr uint32_t AR_IMG = N2MAX * KPAD * 4;   // bytes of one bra-B image (hi or lo) per q
constexpr uint32_t STG_Q = 128 * RMAX;          // floats of one q block of a staging buffer
constexpr uint32_t OFF_KB = 0;
constexpr uint32_t OFF_AR = OFF_KB + KB_STAGES * 2 * KB_IMG;
constexpr uint32_t OFF_STG = OFF_AR + PMAX * 2 * AR_IMG;     // transposer staging: two q blocks of D1
constexpr uint32_t OFF_ESTG = OFF_STG + 2 * STG_Q * 4;       // epilogue staging: one D2 tile
constexpr uint32_t OFF_BAR = OFF_ESTG + STG_Q * 4;
constexpr int CHMAX = 64, PAIRMAX = 64;                    // channel and pair tables kept in shared memory
constexpr uint32_t OFF_TAB = OFF_BAR + 256;                 // block offsets [128], slow-pair offsets [36] (int64)
constexpr uint32_t OFF_META = OFF_TAB + (128 + RMAX) * 8;   // slow-pair staging offsets [36], channels, pair offsets
constexpr uint32_t SW_SMEM = OFF_META + (RMAX + 4 * CHMAX + PAIRMAX + 1) * 4;
static_assert(SW_SMEM <= 227 * 1024, "shared memory");
// tensor-memory columns: D1 | D2 buffers 0,1 | ket A (hi 40 + lo 40) | bra A buffers 0,1. D1 and the
// D2 buffers start on multiples of 32 columns (they are read with 32-column loads), the rest on
// multiples of 16.
constexpr uint32_t TM_D1 = 0, TM_D2 = 160, TM_D2_STRIDE = 64, TM_KA = 272, TM_BA = 352;
constexpr uint32_t TM_COLS = 512;
static_assert(TM_D2 >= N1MAX && TM_D2 + TM_D2_STRIDE + N2MAX <= TM_KA && TM_KA + 2 * KPAD <= TM_BA &&
                  TM_BA + 2 * 2 * KPAD <= TM_COLS, "tensor memory");
static_assert(TM_D2 % 32 == 0 && TM_D2_STRIDE % 32 == 0 && TM_KA % 16 == 0 && TM_BA % 16 == 0 && (2 * KPAD) % 16 == 0,
              "alignment");
constexpr int W_BULK = 0, W_MMA = 1, W_BRA0 = 2, W_KA0 = 4, W_EP0 = 8, W_TR0 = 12;

struct SwArgs {
  int nx, ny, nv, nz, p, nxw, nyw, nvw, nzw, npair;
  const int* ch;         // [nch][4] (x_w, y_w, v_w, z_w), sorted by pair
  const int* pair_off;   // [npair + 1]
  const float* kimg;     // [nch][2][n1p * k1p]
  const float* arimg;    // [p][2][n2p * k2p]
  int n1p, k2p, n2p;     // ket N (q blocks of r2s columns), bra K and N (the ket K is always KPAD)
  int r1, r2, nb;        // rows per block (ket: nx ny, bra: nv nz), blocks per group
  int mw, tw;            // D1 columns of a q block: the first mw (v, z) at q mw, the rest (tw) at p mw + q tw
  int64_t nblk, nk, ngroups;
  const float* in;
  int64_t i_t, i_k, i_X, i_Y;
  float* out;
  int64_t o_t, o_k, o_V, o_Z;
  int v_fast;            // the unit-stride output bundle is V (o_V == 1), else Z: pairs walk its w index innermost
  int* err;
};

// walks the (group, pair) sequence of one CTA. Pairs run with the channel index of the
// output's contiguous bundle innermost, so that consecutive pairs store adjacent runs of
// that bundle while the partly written sectors are still in L2.
struct PairIter {
  int64_t grp;
  int lin, pair;
  const int* off;   // pair offsets (shared-memory copy)
  __device__ void start(const int* pair_off) {
    grp = blockIdx.x;
    lin = -1;
    off = pair_off;
  }
  // next pair (empty ones included); false at the end
  __device__ bool next_any(const SwArgs& a) {
    if (++lin == a.npair) {
      lin = 0;
      grp += gridDim.x;
    }
    pair = a.v_fast ? (lin % a.nvw) * a.nzw + lin / a.nvw : lin;
    return grp < a.ngroups;
  }
  __device__ bool empty(const SwArgs&) const { return off[pair] == off[pair + 1]; }
  __device__ int c0() const { return off[pair]; }
  __device__ int c1() const { return off[pair + 1]; }
  // next pair with at least one channel
  __device__ bool next(const SwArgs& a) {
    while (next_any(a))
      if (!empty(a)) return true;
    return false;
  }
};

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round(__float_as_uint(x));
  lo = tf32_round(__float_as_uint(x - __uint_as_float(hi)));
}

// mma with A from tensor memory, B from a shared-memory descriptor, one CTA
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// waits for this thread's tensor-memory loads, then ties the loaded registers to the wait so
// that no use of them is scheduled before it
template <int N>
__device__ __forceinline__ void tmem_wait_tie(uint32_t (&r)[N]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// named barrier whose participants learn whether all of them passed `ok`
__device__ __forceinline__ bool named_sync_and(int id, int n, bool ok) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// lane 0 waits (sleeping), the warp follows; false on timeout / abort (warp-uniform)
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  bool ok = true;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait_sleep(bar, parity, abort_flag);
  return __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
}

// every MMA issued by this thread has completed (bounded wait; the drain barrier counts one
// commit per issuing thread) before the tensor memory is freed
__device__ __forceinline__ void drain_mmas(uint64_t* drain) {
  mma_commit<false>(drain);
  const unsigned long long t0 = clock64();
  while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_LIMIT) {
  }
}

__global__ void __launch_bounds__(SW_THREADS, 1) k_sandwich_tc(const SwArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bars = (uint64_t*)(smem + OFF_BAR);
  uint64_t* kb_full = bars;                   // [KB_STAGES] ket-B image landed
  uint64_t* kb_empty = kb_full + KB_STAGES;   // [KB_STAGES] its MMAs are done
  uint64_t* ka_full = kb_empty + KB_STAGES;   // ket-A slot written
  uint64_t* ka_empty = ka_full + 1;           // its MMAs are done
  uint64_t* ba_full = ka_empty + 1;           // [2] bra-A buffers
  uint64_t* ba_empty = ba_full + 2;
  uint64_t* d1_full = ba_empty + 2;           // ket accumulator complete / read
  uint64_t* d1_empty = d1_full + 1;
  uint64_t* d2_full = d1_empty + 1;           // both bra accumulator halves complete / read
  uint64_t* d2_empty = d2_full + 1;
  uint64_t* ar_full = d2_empty + 1;
  uint64_t* drain = ar_full + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  float* stg = (float*)(smem + OFF_STG);
  float* estg = (float*)(smem + OFF_ESTG);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (*(volatile int*)a.err) return;   // an earlier launch timed out: nothing is issued

  if (threadIdx.x == 0) {
    for (int s = 0; s < KB_STAGES; ++s) {
      mbar_init(&kb_full[s], 1);
      mbar_init(&kb_empty[s], 1);
    }
    mbar_init(ka_full, 4);
    mbar_init(ka_empty, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&ba_full[s], 4);
      mbar_init(&ba_empty[s], 1);
    }
    mbar_init(d2_full, 2);
    mbar_init(d2_empty, 4);
    mbar_init(d1_full, 1);
    mbar_init(d1_empty, 4);
    mbar_init(ar_full, 1);
    mbar_init(drain, 3);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == W_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // channel and pair tables in shared memory (the 28 KB left to L1 next to this kernel's shared
  // memory would not keep them cached)
  int* s_sstg = (int*)(smem + OFF_META);   // [ns^2] staging offset of the slow pair (epilogue)
  int* s_ch = s_sstg + RMAX;               // [nch][4]
  int* s_poff = s_ch + 4 * CHMAX;          // [npair + 1]
  {
    const int nch = a.pair_off[a.npair];
    for (int i = threadIdx.x; i < 4 * nch; i += blockDim.x) s_ch[i] = a.ch[i];
    for (int i = threadIdx.x; i <= a.npair; i += blockDim.x) s_poff[i] = a.pair_off[i];
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int R1 = a.r1, R2 = a.r2, P = a.p;
  const uint32_t kb_bytes = (uint32_t)a.n1p * KPAD * 4;       // one ket-B image
  const uint32_t ar_bytes = (uint32_t)a.n2p * a.k2p * 4;      // one bra-B image
  int kb_issued = 0;                                          // bulk copies issued (warp 0)

  if (warp == W_BULK) {
    if (lane == 0) {
      bool ok = true;
      mbar_arrive_expect_tx(ar_full, (uint32_t)P * 2 * ar_bytes);
      bulk_g2s(smem + OFF_AR, a.arimg, (uint32_t)P * 2 * ar_bytes, ar_full);
      PairIter pi;
      pi.start(s_poff);
      int it = 0;
      while (ok && pi.next(a)) {
        for (int c = pi.c0(); c < pi.c1(); ++c, ++it) {
          const int st = it % KB_STAGES;
          if (!mbar_wait_sleep(&kb_empty[st], ((it / KB_STAGES) & 1) ^ 1, abort_flag)) { ok = false; break; }
          mbar_arrive_expect_tx(&kb_full[st], 2 * kb_bytes);
          bulk_g2s(smem + OFF_KB + st * 2 * KB_IMG, a.kimg + (int64_t)c * 2 * a.n1p * KPAD, 2 * kb_bytes,
                   &kb_full[st]);
          ++kb_issued;
        }
      }
    }
  } else if (warp == W_MMA) {
    // ket MMAs: the channels of pair k into D1, once the transposer has read pair k - 1
    if (lane == 0) {
      const uint32_t idesc1 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(a.n1p >> 3) << 17) | ((128u >> 4) << 24);
      const uint32_t lbo1 = (uint32_t)(a.n1p / 8) * 128;
      PairIter kp;
      kp.start(s_poff);
      int k = 0, it = 0;
      bool ok = true;
      while (ok && kp.next(a)) {
        if (k > 0 && !mbar_wait(d1_empty, (k - 1) & 1, abort_flag)) break;
        for (int c = kp.c0(); c < kp.c1(); ++c, ++it) {
          const int st = it % KB_STAGES;
          if (!mbar_wait(&kb_full[st], (it / KB_STAGES) & 1, abort_flag) || !mbar_wait(ka_full, it & 1, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint8_t* bh = smem + OFF_KB + st * 2 * KB_IMG;
          const uint8_t* bl = bh + kb_bytes;
          const uint32_t ah = tmem + TM_KA, al = ah + KPAD;
#pragma unroll
          for (int kk = 0; kk < KPAD / 8; ++kk) {
            const uint32_t acc = (c > kp.c0() || kk > 0) ? 1u : 0u;
            mma_ts(tmem + TM_D1, al + kk * 8, sdesc_noswz(bh + 2 * kk * lbo1, lbo1, 128), idesc1, acc);
            mma_ts(tmem + TM_D1, ah + kk * 8, sdesc_noswz(bl + 2 * kk * lbo1, lbo1, 128), idesc1, 1u);
            mma_ts(tmem + TM_D1, ah + kk * 8, sdesc_noswz(bh + 2 * kk * lbo1, lbo1, 128), idesc1, 1u);
          }
          mma_commit<false>(&kb_empty[st]);
          mma_commit<false>(ka_empty);
        }
        if (!ok) break;
        mma_commit<false>(d1_full);
        ++k;
      }
      drain_mmas(drain);
    }
    __syncwarp();
  } else if (warp == W_BRA0 || warp == W_BRA0 + 1) {
    // bra MMAs: warp W_BRA0 + w takes the q blocks that arrive in bra-A slot w (the transposer
    // fills the two slots alternately, so both warps get q blocks of every pair when p >= 2) and
    // accumulates them into D2 half w; the epilogue adds the halves. A tcgen05.mma costs its
    // issuing thread about the same time for any N up to ~200, so two issuers run the narrow
    // (N = 48) bra products at twice the rate of one.
    if (lane == 0) {
      const int w = warp - W_BRA0;
      const uint32_t idesc2 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(a.n2p >> 3) << 17) | ((128u >> 4) << 24);
      const uint32_t lbo2 = (uint32_t)(a.n2p / 8) * 128;
      const int nkk2 = a.k2p / 8;
      const uint32_t ah = tmem + TM_BA + w * 2 * KPAD, al = ah + KPAD;
      const uint32_t d = tmem + TM_D2 + w * TM_D2_STRIDE;
      bool ok = mbar_wait(ar_full, 0, abort_flag);
      PairIter bp;
      bp.start(s_poff);
      int b = 0;
      while (ok && bp.next(a)) {
        if (b > 0 && !mbar_wait(d2_empty, (b - 1) & 1, abort_flag)) break;
        bool first = true;
        for (int q = 0; q < P; ++q) {
          const int qi = P * b + q;   // q blocks run through the two slots in this order
          if ((qi & 1) != w) continue;
          if (!mbar_wait(&ba_full[w], (qi >> 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint8_t* bh = smem + OFF_AR + q * 2 * ar_bytes;
          const uint8_t* bl = bh + ar_bytes;
          for (int kk = 0; kk < nkk2; ++kk) {
            const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
            mma_ts(d, al + kk * 8, sdesc_noswz(bh + 2 * kk * lbo2, lbo2, 128), idesc2, acc);
            mma_ts(d, ah + kk * 8, sdesc_noswz(bl + 2 * kk * lbo2, lbo2, 128), idesc2, 1u);
            mma_ts(d, ah + kk * 8, sdesc_noswz(bh + 2 * kk * lbo2, lbo2, 128), idesc2, 1u);
          }
          mma_commit<false>(&ba_empty[w]);
          first = false;
        }
        if (!ok) break;
        mma_commit<false>(d2_full);
        ++b;
      }
      drain_mmas(drain);
    }
    __syncwarp();
  } else if (warp >= W_KA0 && warp < W_EP0) {
    // ket-A producers: thread = tensor-memory lane = ket row (b, x', y'). The gathers of a channel
    // are issued before waiting for the slot, so they overlap the previous channel's MMAs.
    const int row = (warp % 4) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp % 4) * 32) << 16;
    const int b = row / R1, xy = row % R1, xp = xy / a.ny, yp = xy % a.ny;
    PairIter pr;
    pr.start(s_poff);
    int it = 0;
    bool ok = true;
    int64_t last_grp = -1;
    bool valid = false;
    int64_t base = 0;
    const int64_t sx = (int64_t)a.nxw * a.nx * a.i_X, sy = (int64_t)a.nyw * a.ny * a.i_Y;
    while (ok && pr.next(a)) {
      if (pr.grp != last_grp) {
        last_grp = pr.grp;
        const int64_t blk = pr.grp * a.nb + b;
        valid = b < a.nb && blk < a.nblk;
        if (valid) base = (blk / a.nk) * a.i_t + (blk % a.nk) * a.i_k + xp * a.i_X + yp * a.i_Y;
      }
      for (int c = pr.c0(); c < pr.c1(); ++c, ++it) {
        // ket K index (x, y) -> 6 x + y; columns of absent x or y (edge sites) stay zero
        float v[KPAD];
        if (valid) {
          const int xw = s_ch[4 * c + 0], yw = s_ch[4 * c + 1];
          const float* src = a.in + base + (int64_t)xw * a.nx * a.i_X + (int64_t)yw * a.ny * a.i_Y;
#pragma unroll
          for (int e = 0; e < KPAD; ++e) {
            const int x = e / 6, y = e % 6;
            v[e] = (e < 36 && x < a.nx && y < a.ny) ? __ldg(src + x * sx + y * sy) : 0.f;
          }
        } else {
#pragma unroll
          for (int e = 0; e < KPAD; ++e) v[e] = 0.f;
        }
        if (!warp_wait(ka_empty, (it & 1) ^ 1, abort_flag)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ta = tmem + lane_base + TM_KA;
#pragma unroll
        for (int j = 0; j < KPAD / 8; ++j) {
          uint32_t h[8], l[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) split_tf32(v[j * 8 + e], h[e], l[e]);
          tmem_st8(ta + j * 8, h);
          tmem_st8(ta + KPAD + j * 8, l);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(ka_full);
      }
    }
  } else if (warp >= W_EP0 && warp < W_TR0) {
    // epilogue: D2 -> staging -> output, and the zero pairs. The unit-stride output bundle
    // ("fast": V when o_V = 1, else Z) is stored PEPO-index outermost, so for a fixed block b and
    // slow pair (s, s') the nf^2 elements (f, f') are one contiguous run; a warp stores one run
    // per step, lanes along the run.
    const int row = (warp % 4) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp % 4) * 32) << 16;
    const int tid = threadIdx.x - W_EP0 * 32;   // 0..127
    const int ewarp = warp - W_EP0;
    const bool vf = a.v_fast != 0;
    const int nf = vf ? a.nv : a.nz, ns = vf ? a.nz : a.nv;
    const int nsw = vf ? a.nzw : a.nvw;
    const int64_t o_s = vf ? a.o_Z : a.o_V;
    const int run = nf * nf, ns2 = ns * ns;
    int64_t* blk_base = (int64_t*)(smem + OFF_TAB);   // [nb] output offset of block b of the group
    int64_t* slow_off = blk_base + 128;                // [ns^2] offset of the slow pair (s, s')
    int sf0 = 0, sf1 = 0;                              // staging offsets of this lane's run elements
    {
      const int f0 = lane / nf, f0p = lane % nf, f1 = (lane + 32) / nf, f1p = (lane + 32) % nf;
      sf0 = vf ? (f0 * a.nz * RMAX + f0p * a.nz) : (f0 * RMAX + f0p);
      sf1 = vf ? (f1 * a.nz * RMAX + f1p * a.nz) : (f1 * RMAX + f1p);
    }
    if (tid < ns2) {   // constant over the launch
      const int sx = tid / ns, sxp = tid % ns;
      slow_off[tid] = ((int64_t)sx * nsw * ns + sxp) * o_s;
      s_sstg[tid] = vf ? (sx * RMAX + sxp) : (sx * a.nz * RMAX + sxp * a.nz);   // staging share of (s, s')
    }
    PairIter pr;
    pr.start(s_poff);
    int pn = 0;
    bool ok = true;
    int64_t tab_grp = -1;
    while (ok && pr.next_any(a)) {
      const int64_t blk0 = pr.grp * a.nb;
      const int nbv = (int)min((int64_t)a.nb, a.nblk - blk0);
      if (pr.grp != tab_grp) {   // block offsets of this group
        named_sync(3, 128);      // every thread is done with the previous group's table
        tab_grp = pr.grp;
        if (tid < nbv) {
          const int64_t blk = blk0 + tid;
          blk_base[tid] = (blk / a.nk) * a.o_t + (blk % a.nk) * a.o_k;
        }
        named_sync(3, 128);
      }
      const int pvw = pr.pair / a.nzw, pzw = pr.pair % a.nzw;
      const int fw = vf ? pvw : pzw, sw = vf ? pzw : pvw;
      float* const outp = a.out + (int64_t)fw * run + (int64_t)sw * ns * o_s;
      if (pr.empty(a)) {   // no PEPO channel feeds this output pair: zeros
        for (int bb = 0; bb < nbv; ++bb)
          for (int ss = ewarp; ss < ns2; ss += 4) {
            float* dst = outp + blk_base[bb] + slow_off[ss];
            if (lane < run) dst[lane] = 0.f;
            if (lane + 32 < run) dst[lane + 32] = 0.f;
          }
        continue;
      }
      bool okw = warp_wait(d2_full, pn & 1, abort_flag);
      if (okw) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float4* srow = (float4*)(estg + row * RMAX);
        // the two halves of D2 (the q blocks of bra slot 0 and of slot 1) are added here; each half
        // is read in turn to keep the registers of one half live
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t r2[RMAX];
          const uint32_t t2 = tmem + lane_base + TM_D2 + hh * TM_D2_STRIDE;
          if (R2 > 4) tmem_ld32_async(t2, r2);
          else tmem_ld4(t2, r2);
          if (R2 > 32) tmem_ld4(t2 + 32, r2 + 32);
          tmem_wait_tie(r2);
          if (hh == 1) {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(d2_empty);
          }
#pragma unroll
          for (int j = 0; j < RMAX / 4; ++j)
            if (j * 4 < R2) {
              float4 v = make_float4(__uint_as_float(r2[4 * j]), __uint_as_float(r2[4 * j + 1]),
                                     __uint_as_float(r2[4 * j + 2]), __uint_as_float(r2[4 * j + 3]));
              if (hh == 1) {
                const float4 u = srow[j];
                v.x += u.x;
                v.y += u.y;
                v.z += u.z;
                v.w += u.w;
              }
              srow[j] = v;
            }
        }
      }
      if (!named_sync_and(3, 128, okw)) { ok = false; break; }
      for (int bb = 0; bb < nbv; ++bb)
        for (int ss = ewarp; ss < ns2; ss += 4) {
          // staging row (b, v, z), column (v', z'): the block's and the slow pair's shares
          const int so = bb * R2 * RMAX + s_sstg[ss];
          float* dst = outp + blk_base[bb] + slow_off[ss];
          if (lane < run) dst[lane] = estg[so + sf0];
          if (lane + 32 < run) dst[lane + 32] = estg[so + sf1];
        }
      named_sync(3, 128);   // the staging is free for the next pair
      ++pn;
    }
  } else if (warp >= W_TR0) {
    // transposer: D1 (rows (b, x', y')) -> staging -> bra A (rows (b, v, z), K = (x', y')), two
    // q blocks at a time; D1 is released once its last q block has been read.
    const int row = (warp % 4) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp % 4) * 32) << 16;
    const int bb = row / R2, vz = row % R2;
    const bool rvalid = row < a.nb * R2;
    const float* scol = stg + (bb * R1) * RMAX + vz;   // staging column of this bra row
    PairIter pr;
    pr.start(s_poff);
    int pn = 0, qi = 0;
    bool ok = true;
    while (ok && pr.next(a)) {
      bool okw = warp_wait(d1_full, pn & 1, abort_flag);
      for (int q0 = 0; q0 < P && ok; q0 += 2) {
        const int nq = min(2, P - q0);
        if (okw) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int h = 0; h < nq; ++h) {
            uint32_t r[RMAX];
            const int q = q0 + h;
            const uint32_t tq = tmem + lane_base + TM_D1;
            if (a.mw == 32) {
              tmem_ld32_async(tq + q * 32, r);
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (j * 4 < a.mw) tmem_ld4(tq + q * a.mw + j * 4, r + j * 4);
            }
            if (a.tw > 0) tmem_ld4(tq + P * a.mw + q * a.tw, r + 32);
            tmem_wait_tie(r);
            float4* srow = (float4*)(stg + h * STG_Q + row * RMAX);
#pragma unroll
            for (int j = 0; j < RMAX / 4; ++j)
              if (j * 4 < R2)
                srow[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                      __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
          }
          if (q0 + nq == P) {   // the whole of D1 has been read
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(d1_empty);
          }
        }
        if (!named_sync_and(2, 128, okw)) { ok = false; break; }
        for (int h = 0; h < nq && okw; ++h, ++qi) {
          float v[KPAD];
#pragma unroll
          for (int e = 0; e < KPAD; ++e) v[e] = (rvalid && e < R1) ? scol[h * STG_Q + e * RMAX] : 0.f;
          if (!warp_wait(&ba_empty[qi & 1], ((qi >> 1) & 1) ^ 1, abort_flag)) { okw = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ta = tmem + lane_base + TM_BA + (qi & 1) * 2 * KPAD;
#pragma unroll
          for (int j = 0; j < KPAD / 8; ++j) {
            if (j * 8 < a.k2p) {
              uint32_t hh[8], ll[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) split_tf32(v[j * 8 + e], hh[e], ll[e]);
              tmem_st8(ta + j * 8, hh);
              tmem_st8(ta + KPAD + j * 8, ll);
            }
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&ba_full[qi & 1]);
        }
        // every warp is done with the staging before the next q blocks overwrite it
        if (!named_sync_and(2, 128, okw)) { ok = false; break; }
      }
      ++pn;
    }
  }

  // every role has left its loop once all threads meet here
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag) {
    if (warp == W_BULK && lane == 0) {   // wait (bounded) for bulk copies still in flight
      for (int it = kb_issued > KB_STAGES ? kb_issued - KB_STAGES : 0; it < kb_issued; ++it) {
        const int st = it % KB_STAGES;
        const unsigned long long t0 = clock64();
        while (!mbar_try_wait(&kb_full[st], (it / KB_STAGES) & 1) && clock64() - t0 < WAIT_LIMIT) {
        }
      }
      const unsigned long long t0 = clock64();
      while (!mbar_try_wait(ar_full, 0) && clock64() - t0 < WAIT_LIMIT) {
      }
    }
    if (threadIdx.x == 0) atomicExch(a.err, 1);
  }
  __syncthreads();
  if (warp == W_MMA) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM_COLS));
  }
}

// hi/lo operand images in the K-major no-swizzle layout of the MMA: element (n, k) of an
// n_rows x k_cols image at (k / 4) * (n_rows / 8) * 32 + (n / 8) * 32 + (n % 8) * 4 + k % 4
__device__ __forceinline__ int64_t img_off(int n, int k, int n_rows) {
  return (int64_t)(k / 4) * (n_rows / 8) * 32 + (n / 8) * 32 + (n % 8) * 4 + (k % 4);
}

// ket images: channel c, k = 6 x + y (zero outside the site's x, y), rows n in the column order
// of D1: (q, vz) at q mw + vz for vz < mw, at p mw + q tw + vz - mw for the rest; value
// AW_c[x][y][v][z][q]
__global__ void k_ket_images(const float* aw, int nch, int nx, int ny, int nv, int nz, int p, int mw, int tw,
                             int n1p, float* img) {
  const int R2 = nv * nz;
  const int64_t per = (int64_t)n1p * KPAD;
  const int64_t tot = per * nch;
  const int64_t wsz = (int64_t)nx * ny * R2 * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / per);
    const int n = (int)((e % per) / KPAD), k = (int)(e % KPAD);
    int q, vz;
    if (n < p * mw) {
      q = n / mw;
      vz = n % mw;
    } else {
      q = tw > 0 ? (n - p * mw) / tw : p;
      vz = tw > 0 ? mw + (n - p * mw) % tw : R2;
    }
    const int x = k / 6, y = k % 6;
    float v = 0.f;
    if (q < p && vz < R2 && k < 36 && x < nx && y < ny) v = aw[c * wsz + ((int64_t)(x * ny + y) * R2 + vz) * p + q];
    uint32_t h, l;
    split_tf32(v, h, l);
    float* base = img + (int64_t)c * 2 * per;
    base[img_off(n, k, n1p)] = __uint_as_float(h);
    base[per + img_off(n, k, n1p)] = __uint_as_float(l);
  }
}

// bra images: q, n = (v', z'), k = (x', y') = x' ny + y'; value A[x'][y'][v'][z'][q]
__global__ void k_bra_images(const float* ar, int nx, int ny, int nv, int nz, int p, int n2p, int k2p, float* img) {
  const int R1 = nx * ny, R2 = nv * nz;
  const int64_t per = (int64_t)n2p * k2p;
  const int64_t tot = per * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / per);
    const int n = (int)((e % per) / k2p), k = (int)(e % k2p);
    float v = 0.f;
    if (n < R2 && k < R1) v = ar[((int64_t)k * R2 + n) * p + q];
    uint32_t h, l;
    split_tf32(v, h, l);
    float* base = img + (int64_t)q * 2 * per;
    base[img_off(n, k, n2p)] = __uint_as_float(h);
    base[per + img_off(n, k, n2p)] = __uint_as_float(l);
  }
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct TcShape {
  int r1, r2, mw, tw, n1p, k2p, n2p;
};
TcShape tc_shape(const SandOrient& o) {
  TcShape t;
  t.r1 = o.nx * o.ny;
  t.r2 = o.nv * o.nz;
  t.mw = t.r2 >= 32 ? 32 : round_up(t.r2, 4);
  t.tw = round_up(std::max(t.r2 - 32, 0), 4);
  t.n1p = round_up(o.p * (t.mw + t.tw), 16);
  t.k2p = round_up(t.r1, 8);
  t.n2p = round_up(t.r2, 16);
  return t;
}

}  // namespace

bool sandwich_tc_fits(const SandOrient& o) {
  const TcShape t = tc_shape(o);
  return o.nch >= 1 && o.nch <= CHMAX && o.nvw * o.nzw <= PAIRMAX && o.p >= 2 && o.p <= PMAX && o.nx >= 1 && o.ny >= 1 && o.nv >= 1 && o.nz >= 1 && o.nx <= 6 &&
         o.ny <= 6 && o.nv <= 6 && o.nz <= 6 && t.r1 <= RMAX && t.r2 <= RMAX && t.n1p <= N1MAX && t.k2p <= KPAD &&
         t.n2p <= N2MAX;
}

void sandwich_tc_image_floats(const SandOrient& o, size_t* ket, size_t* bra) {
  const TcShape t = tc_shape(o);
  *ket = (size_t)o.nch * 2 * t.n1p * KPAD;
  *bra = (size_t)o.p * 2 * t.n2p * t.k2p;
}

void sandwich_tc_images(cudaStream_t s, const SandOrient& o, float* ket_img, float* bra_img) {
  const TcShape t = tc_shape(o);
  const int64_t nk = (int64_t)o.nch * t.n1p * KPAD, nb = (int64_t)o.p * t.n2p * t.k2p;
  k_ket_images<<<(unsigned)std::min<int64_t>((nk + 255) / 256, 4096), 256, 0, s>>>(
      (const float*)o.d_aw, o.nch, o.nx, o.ny, o.nv, o.nz, o.p, t.mw, t.tw, t.n1p, ket_img);
  FP_LAUNCH();
  k_bra_images<<<(unsigned)std::min<int64_t>((nb + 255) / 256, 4096), 256, 0, s>>>(
      (const float*)o.d_ar, o.nx, o.ny, o.nv, o.nz, o.p, t.n2p, t.k2p, bra_img);
  FP_LAUNCH();
}

void sandwich_apply_tcgen05(cudaStream_t s, const SandOrient& o, int64_t nt, int64_t nk, const float* in,
                            int64_t i_t, int64_t i_k, int64_t i_X, int64_t i_Y, float* out, int64_t o_t, int64_t o_k,
                            int64_t o_V, int64_t o_Z, int* err) {
  if (nt <= 0 || nk <= 0) return;
  FP_CHECK(sandwich_tc_fits(o) && o.d_kimg && o.d_arimg, FPEPS_ERR_UNSUPPORTED,
           "tcgen05 sandwich: site dimensions out of range");
  FP_CHECK(((uintptr_t)o.d_kimg % 16) == 0 && ((uintptr_t)o.d_arimg % 16) == 0, FPEPS_ERR_ARG,
           "tcgen05 sandwich: image alignment");
  FP_CHECK(o.nch <= CHMAX && o.nvw * o.nzw <= PAIRMAX, FPEPS_ERR_UNSUPPORTED, "tcgen05 sandwich: too many channels");
  SwArgs a;
  a.nx = o.nx; a.ny = o.ny; a.nv = o.nv; a.nz = o.nz; a.p = o.p;
  a.nxw = o.nxw; a.nyw = o.nyw; a.nvw = o.nvw; a.nzw = o.nzw;
  a.npair = o.nvw * o.nzw;
  a.ch = o.d_ch;
  a.pair_off = o.d_pair_off;
  a.kimg = (const float*)o.d_kimg;
  a.arimg = (const float*)o.d_arimg;
  const TcShape t = tc_shape(o);
  a.r1 = t.r1;
  a.r2 = t.r2;
  a.mw = t.mw;
  a.tw = t.tw;
  a.n1p = t.n1p;
  a.k2p = t.k2p;
  a.n2p = t.n2p;
  a.nb = 128 / std::max(a.r1, a.r2);
  a.nblk = nt * nk;
  a.nk = nk;
  a.ngroups = (a.nblk + a.nb - 1) / a.nb;
  a.in = in; a.i_t = i_t; a.i_k = i_k; a.i_X = i_X; a.i_Y = i_Y;
  a.out = out; a.o_t = o_t; a.o_k = o_k; a.o_V = o_V; a.o_Z = o_Z;
  a.v_fast = o_V == 1 ? 1 : 0;   // the same rule as bundle_index's callers: V when it has unit stride
  a.err = err;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    FP_CUDA(cudaGetDevice(&dev));
    FP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  static bool attr = false;
  if (!attr) {
    FP_CUDA(cudaFuncSetAttribute(k_sandwich_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SW_SMEM));
    attr = true;
  }
  const int64_t grid = std::min<int64_t>(a.ngroups, sms);
  k_sandwich_tc<<<(unsigned)grid, SW_THREADS, SW_SMEM, s>>>(a);
  FP_LAUNCH();
}

}  // namespace fpeps
