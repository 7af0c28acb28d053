// Randomized-SVD building blocks (Sec. IV; Halko et al. 2011, Example 1.6):
// the Gaussian sketch Omega, FP64 Gram matrices, Cholesky QR, the one-sided
// Jacobi SVD of small matrices, norms and layout helpers.
//
// Gaussian sketch: Philox4x64-10 (Salmon et al., SC'11) keyed by (seed, layer)
// with counter (i >> 1, j, site | stage << 16, row | env << 16); the word pair
// (x0,x1) for even i and (x2,x3) for odd i gives u = ((x >> 11) + 0.5) 2^-53
// and z = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller). i is the flat row index of
// the sketched space in C order of its (bond, bundle) legs.
//
// One-sided Jacobi SVD: Hestenes' method with the cyclic round-robin ordering;
// each rotation makes two columns orthogonal (Demmel and Veselic 1992). The
// path always applies it to the transposed triangular factor of a QR (the
// preconditioned form of Drmac and Veselic 2008), where it converges in about
// ten sweeps; the sweep count is capped at 30.
#include <cstdio>
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace fpeps {
namespace {

constexpr uint64_t PH_M0 = 0xD2E7470EE14C6C93ull, PH_M1 = 0xCA5A826395121157ull;
constexpr uint64_t PH_W0 = 0x9E3779B97F4A7C15ull, PH_W1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(PH_M0, c[0]), lo0 = PH_M0 * c[0];
    uint64_t hi1 = __umul64hi(PH_M1, c[2]), lo1 = PH_M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += PH_W0; k1 += PH_W1;
  }
}

__device__ __forceinline__ double u53(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }

// memory position pos = hi * lo_dim + lo within a column; canonical flat index
// i = lo * hi_dim + hi when swap != 0, else i = pos.
template <class T>
__global__ void k_sketch(T* out, int64_t n_rows, int64_t k, int64_t ld, int64_t hi_dim, int64_t lo_dim, int swap,
                         uint64_t seed, uint64_t layer, uint64_t w2, uint64_t w3) {
  const int64_t n = n_rows * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = e / n_rows, pos = e % n_rows;
    int64_t i = swap ? (pos % lo_dim) * hi_dim + pos / lo_dim : pos;
    uint64_t c[4] = {(uint64_t)i >> 1, (uint64_t)j, w2, w3};
    philox4x64(c, seed, layer);
    uint64_t a = (i & 1) ? c[2] : c[0];
    uint64_t b = (i & 1) ? c[3] : c[1];
    double z = sqrt(-2.0 * log(u53(a))) * cospi(2.0 * u53(b));
    out[j * ld + pos] = (T)z;
  }
}

// G[i][j] += sum_r Y[i*ld + r] * Y[j*ld + r] over one row chunk; 32x32 tile per block.
template <class T>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ Y, int64_t m, int64_t k, int64_t ld,
                                              int64_t chunk, double* G) {
  __shared__ double si[32][33];
  __shared__ double sj[32][33];
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj < ti) return;   // upper tiles only, mirrored at the end
  const int64_t r0 = blockIdx.z * chunk, r1 = min(m, r0 + chunk);
  const int tid = threadIdx.x;
  const int li = tid / 8, lj = (tid % 8) * 4;   // each thread: 1 row x 4 cols of the tile
  double acc[4] = {0, 0, 0, 0};
  for (int64_t rb = r0; rb < r1; rb += 32) {
    for (int e = tid; e < 32 * 32; e += 256) {
      int c = e / 32, rr = e % 32;
      int64_t r = rb + rr;
      int64_t ci = (int64_t)ti * 32 + c, cj = (int64_t)tj * 32 + c;
      si[c][rr] = (r < r1 && ci < k) ? (double)Y[ci * ld + r] : 0.0;
      sj[c][rr] = (r < r1 && cj < k) ? (double)Y[cj * ld + r] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      double a = si[li][rr];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(a, sj[lj + q][rr], acc[q]);
    }
    __syncthreads();
  }
  int64_t gi = (int64_t)ti * 32 + li;
  if (gi >= k) return;
  for (int q = 0; q < 4; ++q) {
    int64_t gj = (int64_t)tj * 32 + lj + q;
    if (gj >= k || gj < gi) continue;
    atomicAdd(&G[gi * k + gj], acc[q]);
  }
}

// FP64-class Gram of FP32 data on the FP32 pipes. Each product a*b is split
// exactly into p + e (p = fl(a*b), e = fma(a, b, -p)); p is accumulated with
// an error-free two-sum into (hi, lo) and e is added to lo (double-float
// summation: Dekker 1971; Ogita, Rump and Oishi 2005). Each 64x64 tile of an
// upper block of G is summed over one row chunk and added to G in FP64.
__device__ __forceinline__ void df_add_prod(float a, float b, float& hi, float& lo) {
  const float p = a * b;
  const float e = fmaf(a, b, -p);
  const float s = hi + p;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (p - bp);
  hi = s;
  lo += err + e;
}

__global__ void __launch_bounds__(256) k_gram_df(const float* __restrict__ Y, int64_t m, int64_t k, int64_t ld,
                                                 int64_t chunk, double* G) {
  __shared__ float si[16][65];
  __shared__ float sj[16][65];
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (tj < ti) return;
  const int64_t r0 = blockIdx.z * chunk, r1 = min(m, r0 + chunk);
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;   // 4x4 outputs: rows tr + 16 a, cols tc + 16 b
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { hi[a][b] = 0.f; lo[a][b] = 0.f; }
  for (int64_t rb = r0; rb < r1; rb += 16) {
    for (int e = tid; e < 16 * 64; e += 256) {
      int c = e / 16, rr = e % 16;
      int64_t r = rb + rr;
      int64_t ci = (int64_t)ti * 64 + c, cj = (int64_t)tj * 64 + c;
      si[rr][c] = (r < r1 && ci < k) ? Y[ci * ld + r] : 0.f;
      sj[rr][c] = (r < r1 && cj < k) ? Y[cj * ld + r] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 16; ++rr) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = si[rr][tr + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = sj[rr][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) df_add_prod(av[a], bv[b], hi[a][b], lo[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int64_t gi = (int64_t)ti * 64 + tr + 16 * a;
    if (gi >= k) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int64_t gj = (int64_t)tj * 64 + tc + 16 * b;
      if (gj >= k || gj < gi) continue;
      atomicAdd(&G[gi * k + gj], (double)hi[a][b] + (double)lo[a][b]);
    }
  }
}

__global__ void k_mirror_upper(double* G, int k) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)k * k; e += (int64_t)gridDim.x * blockDim.x) {
    int i = e / k, j = e % k;
    if (j < i) G[e] = G[(int64_t)j * k + i];
  }
}

// In-place Cholesky G = R^T R (R upper, row-major), one block, for the Gram
// matrix of the columns of Y. A pivot at or below tol * max diag means column j
// depends numerically on the columns before it: row j of R is set to zero (the
// column of Q it would give is zero). info = 1 only for non-finite input.
__global__ void __launch_bounds__(1024) k_cholesky(double* G, int k, double tol, int* info) {
  __shared__ double piv_s;
  __shared__ double dmax_s;
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) {
    double dm = 0;
    bool fin = true;
    for (int i = 0; i < k; ++i) {
      const double d = G[(int64_t)i * k + i];
      fin = fin && isfinite(d);
      dm = fmax(dm, d);
    }
    dmax_s = dm;
    bad = !fin;
  }
  __syncthreads();
  if (bad) { if (tid == 0) info[0] = 1; return; }
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double d = G[(int64_t)j * k + j];
      if (!isfinite(d)) bad = 1;
      piv_s = d > tol * dmax_s ? sqrt(d) : 0.0;
      G[(int64_t)j * k + j] = piv_s;
    }
    __syncthreads();
    if (bad) { if (tid == 0) info[0] = 1; return; }
    const double piv = piv_s;
    for (int c = j + 1 + tid; c < k; c += blockDim.x) G[(int64_t)j * k + c] = piv > 0 ? G[(int64_t)j * k + c] / piv : 0.0;
    __syncthreads();
    const int n = k - j - 1;
    // trailing update of the upper triangle: G[i][c] -= R[j][i] R[j][c], i <= c
    for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) {
      int i = j + 1 + (int)(e / n), c = j + 1 + (int)(e % n);
      if (c >= i) G[(int64_t)i * k + c] -= G[(int64_t)j * k + i] * G[(int64_t)j * k + c];
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)k * k; e += blockDim.x) {
    int i = e / k, c = e % k;
    if (c < i) G[e] = 0.0;
  }
  if (tid == 0) info[0] = 0;
}

// Blocked right-looking Cholesky over the whole GPU (cooperative launch, panel
// width 32): block 0 factors the diagonal block in shared memory, every block
// solves its share of the panel row, every block updates its share of the
// trailing upper triangle; grid barriers in between. Same pivot rule as above.
constexpr int CH_NB = 32;
__global__ void __launch_bounds__(256) k_cholesky_coop(double* G, int k, double tol, int* info, double* ws) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double D[CH_NB][CH_NB + 1];
  __shared__ double inv_s[CH_NB];
  __shared__ double rinv_s;
  __shared__ int bad_s;
  const int tid = threadIdx.x;
  const int lane = tid % 32, warp = tid / 32;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + tid;
  const int64_t gsize = (int64_t)gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && tid == 0) {
    double dm = 0;
    bool fin = true;
    for (int i = 0; i < k; ++i) {
      const double d = G[(int64_t)i * k + i];
      fin = fin && isfinite(d);
      dm = fmax(dm, d);
    }
    ws[0] = dm;
    info[0] = !fin;
  }
  grid.sync();
  if (*(volatile int*)info) return;
  const double dmax = ws[0];
  for (int p0 = 0; p0 < k; p0 += CH_NB) {
    const int nb = min(CH_NB, k - p0);
    if (blockIdx.x == 0) {
      for (int e = tid; e < nb * nb; e += blockDim.x) D[e / nb][e % nb] = G[(int64_t)(p0 + e / nb) * k + p0 + e % nb];
      if (tid == 0) bad_s = 0;
      __syncthreads();
      for (int j = 0; j < nb; ++j) {
        // FP64 sqrt and division are long latencies here (~680 / ~430 cycles): the pivot's
        // sqrt and the row's scale factor rsqrt run side by side
        if (tid == 0) {
          const double d = D[j][j];
          if (!isfinite(d)) bad_s = 1;
          const bool keep = d > tol * dmax;
          D[j][j] = keep ? sqrt(d) : 0.0;
          rinv_s = keep ? rsqrt(d) : 0.0;
        }
        __syncthreads();
        if (bad_s) break;
        for (int c = j + 1 + tid; c < nb; c += blockDim.x) D[j][c] *= rinv_s;
        __syncthreads();
        const int n = nb - j - 1;
        for (int e = tid; e < n * n; e += blockDim.x) {
          int i = j + 1 + e / n, c = j + 1 + e % n;
          if (c >= i) D[i][c] -= D[j][i] * D[j][c];
        }
        __syncthreads();
      }
      if (tid == 0 && bad_s) info[0] = 1;
      for (int e = tid; e < nb * nb; e += blockDim.x) {
        int i = e / nb, c = e % nb;
        if (c >= i) G[(int64_t)(p0 + i) * k + p0 + c] = D[i][c];
      }
    }
    grid.sync();
    if (*(volatile int*)info) return;
    // panel row: R[p0:p0+nb, c] solves R_pp^T x = G[p0:p0+nb, c] for c >= p0 + nb, one warp
    // per column spread over the whole grid (lane i holds row i; each solved value is
    // broadcast and folded into the rows below it), every block with the factored diagonal
    // block and its pivots' reciprocals in shared memory
    for (int e = tid; e < nb * nb; e += blockDim.x) D[e / nb][e % nb] = G[(int64_t)(p0 + e / nb) * k + p0 + e % nb];
    __syncthreads();
    for (int i = tid; i < nb; i += blockDim.x) inv_s[i] = D[i][i] > 0 ? 1.0 / D[i][i] : 0.0;
    __syncthreads();
    {
      const int wpb = blockDim.x / 32;
      for (int64_t c = p0 + nb + (int64_t)blockIdx.x * wpb + warp; c < k; c += (int64_t)gridDim.x * wpb) {
        const double gl = lane < nb ? G[(int64_t)(p0 + lane) * k + c] : 0.0;
        double acc = 0.0, mine = 0.0;
        for (int l = 0; l < nb; ++l) {
          double r = 0.0;
          if (lane == l) r = inv_s[l] != 0.0 ? (gl - acc) * inv_s[l] : 0.0;
          r = __shfl_sync(0xffffffffu, r, l);
          if (lane == l) mine = r;
          if (lane > l && lane < nb) acc = fma(D[l][lane], r, acc);
        }
        if (lane < nb) G[(int64_t)(p0 + lane) * k + c] = mine;
      }
    }
    grid.sync();
    // trailing update of the upper triangle (four partial sums: the dependent FP64 FMA
    // chain is 64 cycles per step)
    const int64_t r0 = p0 + nb, n = k - r0;
    for (int64_t e = gtid; e < n * n; e += gsize) {
      const int64_t i = r0 + e / n, c = r0 + e % n;
      if (c < i) continue;
      double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      int l = 0;
      for (; l + 4 <= nb; l += 4) {
        a0 = fma(G[(int64_t)(p0 + l) * k + i], G[(int64_t)(p0 + l) * k + c], a0);
        a1 = fma(G[(int64_t)(p0 + l + 1) * k + i], G[(int64_t)(p0 + l + 1) * k + c], a1);
        a2 = fma(G[(int64_t)(p0 + l + 2) * k + i], G[(int64_t)(p0 + l + 2) * k + c], a2);
        a3 = fma(G[(int64_t)(p0 + l + 3) * k + i], G[(int64_t)(p0 + l + 3) * k + c], a3);
      }
      for (; l < nb; ++l) a0 = fma(G[(int64_t)(p0 + l) * k + i], G[(int64_t)(p0 + l) * k + c], a0);
      G[i * k + c] -= (a0 + a1) + (a2 + a3);
    }
    grid.sync();
  }
  for (int64_t e = gtid; e < (int64_t)k * k; e += gsize) {
    int64_t i = e / k, c = e % k;
    if (c < i) G[e] = 0.0;
  }
}

// Rinv = R^{-1} for upper-triangular R (row-major): one warp per column, the
// back-substitution dot products split over the lanes, the column kept in
// shared memory. Rows of R with a zero diagonal (dependent columns) give zero
// rows and columns of Rinv: the inverse of the non-zero part, padded with zeros.
__global__ void __launch_bounds__(128) k_tri_inverse_warp(const double* R, int k, double* Rinv) {
  extern __shared__ double xs_all[];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  double* x = xs_all + (int64_t)w * k;
  const int j = blockIdx.x * (blockDim.x / 32) + w;
  if (j >= k) return;
  for (int i = lane; i < k; i += 32) x[i] = 0.0;
  __syncwarp();
  const double rjj = R[(int64_t)j * k + j];
  if (rjj != 0.0) {
    if (lane == 0) x[j] = 1.0 / rjj;
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
      const double rii = R[(int64_t)i * k + i];
      if (rii == 0.0) continue;   // x[i] stays zero
      double sdot = 0;
      for (int l = i + 1 + lane; l <= j; l += 32) sdot = fma(R[(int64_t)i * k + l], x[l], sdot);
      for (int o = 16; o; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
      if (lane == 0) x[i] = -sdot / rii;
      __syncwarp();
    }
  }
  __syncwarp();
  for (int i = lane; i < k; i += 32) Rinv[(int64_t)i * k + j] = x[i];
}

// One round of the one-sided Jacobi method on the columns of M (col-major,
// k x k) with the accumulated right rotations in V. Pairs of the round-robin
// schedule: player positions 0..kk-1 (kk even), position 0 fixed.
__device__ __forceinline__ int rr_player(int pos, int round, int kk) {
  if (pos == 0) return 0;
  return 1 + ((pos - 1 + round) % (kk - 1));
}

__global__ void __launch_bounds__(1024) k_jacobi_svd(double* M, double* V, int k, int max_sweeps, double eps,
                                                      int* info) {
  const int kk = (k % 2) ? k + 1 : k;   // dummy column k when odd
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
  __shared__ int rotated;
  __shared__ double fro2;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) V[e] = ((e / k) == (e % k)) ? 1.0 : 0.0;
  if (threadIdx.x == 0) {
    double f = 0;
    for (int64_t e = 0; e < (int64_t)k * k; ++e) f = fma(M[e], M[e], f);
    fro2 = f;
  }
  __syncthreads();
  // a column whose squared norm is below 1e-30 of the whole matrix carries no
  // resolvable direction: rotations against it only stir rounding noise
  const double tiny = 1e-30 * fro2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < kk - 1; ++round) {
      for (int pr = warp; pr < kk / 2; pr += nwarp) {
        int a = rr_player(pr, round, kk), b = rr_player(kk - 1 - pr, round, kk);
        int p = min(a, b), q = max(a, b);
        if (q >= k) continue;
        double* mp = M + (int64_t)p * k;
        double* mq = M + (int64_t)q * k;
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < k; i += 32) {
          double x = mp[i], y = mq[i];
          al = fma(x, x, al); be = fma(y, y, be); ga = fma(x, y, ga);
        }
        for (int o = 16; o; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (ga == 0.0 || fmin(al, be) <= tiny || fabs(ga) <= eps * sqrt(al) * sqrt(be)) continue;
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int i = lane; i < k; i += 32) {
          double x = mp[i], y = mq[i];
          mp[i] = c * x - s * y;
          mq[i] = s * x + c * y;
          double vx = V[(int64_t)p * k + i], vy = V[(int64_t)q * k + i];
          V[(int64_t)p * k + i] = c * vx - s * vy;
          V[(int64_t)q * k + i] = s * vx + c * vy;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  // reaching the sweep cap leaves the columns orthogonal to rounding level; it is not an error
  if (threadIdx.x == 0) info[0] = 0;
}

// The same method spread over the whole GPU, in blocks of two columns (block b:
// columns 2b and 2b + 1). A round-robin schedule over the blocks gives every CTA a
// pair of blocks (A, B) per round; the CTA copies their four columns of M and of V to
// shared memory and rotates the four cross pairs, two at a time ((a0,b0) (a1,b1), then
// (a0,b1) (a1,b0)), after first rotating each block's own pair in the first round of a
// sweep. Every column pair is visited once per sweep, as in the scalar cyclic order,
// with one grid barrier per round of blocks. Each rotation is carried by two warps (one
// half of the rows each, partial dot products exchanged in shared memory), so the four
// warps of a CTA keep all four FP64 pipes of the SM busy: FP64 is the limit here (~2 FMA
// per cycle per SM on this part; a rotation of two length-k columns of M and of V costs
// ~11 k FMA).
// ws[0..1]: sweep rotation counters (two, alternating), ws[2]: squared Frobenius norm,
// ws[3]: sweeps used, ws[4..5]: counters of rotations above sqrt(big2) (alternating).
constexpr int JB_THREADS = 128;

// rotation of local columns (p, q) by the two warps h = 0, 1 of a pair slot: rows
// [h * half, (h + 1) * half); part[6] holds the two halves' (alpha, beta, gamma)
// *big (if given) is set when the rotation's |gamma| / sqrt(alpha beta) exceeds sqrt(big2)
__device__ __forceinline__ bool jacobi_rotate_split(double* __restrict__ mp, double* __restrict__ mq,
                                                    double* __restrict__ vp, double* __restrict__ vq, int k, int h,
                                                    int lane, double* part, double eps, double tiny, bool* big,
                                                    double big2) {
  const int half = (k + 1) / 2, i0 = h * half, i1 = min(k, i0 + half);
  double al = 0, be = 0, ga = 0;
  for (int i = i0 + lane; i < i1; i += 32) {
    const double x = mp[i], y = mq[i];
    al = fma(x, x, al);
    be = fma(y, y, be);
    ga = fma(x, y, ga);
  }
  for (int o = 16; o; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (lane == 0) {
    part[3 * h + 0] = al;
    part[3 * h + 1] = be;
    part[3 * h + 2] = ga;
  }
  __syncthreads();
  // both warps add the halves in the same order, so they take the same decision and angle
  al = part[0] + part[3];
  be = part[1] + part[4];
  ga = part[2] + part[5];
  // |gamma| <= eps sqrt(alpha beta) tested squared: FP64 sqrt and division are long serial
  // latencies here (~680 and ~430 cycles), so the angle takes one of each plus one rsqrt:
  // tan = sign(d) 2 gamma / (|d| + sqrt(d^2 + 4 gamma^2)), d = beta - alpha, which is
  // sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) with zeta = d / (2 gamma)
  const bool rot = !(ga == 0.0 || fmin(al, be) <= tiny || ga * ga <= eps * eps * al * be);
  if (rot) {
    if (big && ga * ga > big2 * al * be) *big = true;
    const double d = be - al, g2 = 2.0 * ga;
    const double t = (d >= 0 ? g2 : -g2) / (fabs(d) + sqrt(fma(d, d, g2 * g2)));
    const double c = rsqrt(fma(t, t, 1.0)), sn = c * t;
    for (int i = i0 + lane; i < i1; i += 32) {
      const double x = mp[i], y = mq[i], a = vp[i], b = vq[i];
      mp[i] = c * x - sn * y;
      mq[i] = sn * x + c * y;
      vp[i] = c * a - sn * b;
      vq[i] = sn * a + c * b;
    }
  }
  return rot;
}

__global__ void __launch_bounds__(JB_THREADS) k_jacobi_svd_blk(double* M, double* V, int k, int max_sweeps,
                                                                double eps, double big2, unsigned long long* ws) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double jsh[];   // M columns [4][k], V columns [4][k], partial dots [2][6]
  double* sm = jsh;
  double* sv = jsh + 4 * (int64_t)k;
  double* part = jsh + 8 * (int64_t)k;
  const int nb = (k + 1) / 2, nbe = nb + (nb & 1);   // blocks; a dummy block when nb is odd
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int slot = warp / 2, h = warp % 2;           // pair slot and row half of this warp
  double* fro2p = (double*)&ws[2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)k * k; e += (int64_t)gridDim.x * blockDim.x)
    V[e] = ((e / k) == (e % k)) ? 1.0 : 0.0;
  if (blockIdx.x == 0) {   // ||M||_F^2 by block 0
    __shared__ double red[JB_THREADS / 32];
    double f = 0;
    for (int64_t e = threadIdx.x; e < (int64_t)k * k; e += blockDim.x) f = fma(M[e], M[e], f);
    for (int o = 16; o; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) red[warp] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0;
      for (int w = 0; w < JB_THREADS / 32; ++w) t += red[w];
      *fro2p = t;
      ws[0] = ws[1] = ws[4] = ws[5] = 0;
    }
  }
  grid.sync();
  const double tiny = 1e-30 * (*fro2p);
  // The rotation counter of sweep s lives in ws[s & 1] (its count of rotations above
  // sqrt(big2) in ws[4 + (s & 1)]); every block reads it after the last
  // round and a further barrier follows, so all blocks take the same break decision; the slot
  // is cleared for sweep s+2 at round 1 of sweep s+1, after those reads.
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < nbe - 1; ++round) {
      if (round == 1 && blockIdx.x == 0 && threadIdx.x == 0) ws[(sweep + 1) & 1] = ws[4 + ((sweep + 1) & 1)] = 0;
      const int A = rr_player((int)blockIdx.x, round, nbe), B = rr_player(nbe - 1 - (int)blockIdx.x, round, nbe);
      // local columns 0, 1 (block A) and 2, 3 (block B); -1: absent
      int col[4];
      col[0] = 2 * A;
      col[1] = 2 * A + 1;
      col[2] = 2 * B;
      col[3] = 2 * B + 1;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (col[j] >= k) col[j] = -1;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
          const bool in = col[j] >= 0;
          sm[j * k + i] = in ? M[(int64_t)col[j] * k + i] : 0.0;
          sv[j * k + i] = in ? V[(int64_t)col[j] * k + i] : 0.0;
        }
      __syncthreads();
      int nrot = 0;
      bool big = false;
      // inner rounds: the blocks' own pairs (first round of a sweep), then the cross pairs
      // inner round 0: (0,1) (2,3); 1: (0,2) (1,3); 2: (0,3) (1,2) -- slot 0 takes the first pair
      for (int ir = round == 0 ? 0 : 1; ir < 3; ++ir) {
        const int p = ir == 0 ? 2 * slot : slot;
        const int q = ir == 0 ? 2 * slot + 1 : (ir == 1 ? slot + 2 : 3 - slot);
        double* pt = part + 6 * slot;
        if (col[p] >= 0 && col[q] >= 0) {
          if (jacobi_rotate_split(sm + p * k, sm + q * k, sv + p * k, sv + q * k, k, h, lane, pt, eps, tiny, &big,
                                  big2))
            ++nrot;
        } else {
          __syncthreads();   // the same barrier count as a rotating slot
        }
        __syncthreads();
      }
      if (h == 0 && lane == 0 && nrot) atomicAdd(&ws[sweep & 1], (unsigned long long)nrot);
      if (h == 0 && lane == 0 && big) atomicAdd(&ws[4 + (sweep & 1)], 1ull);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (col[j] >= 0)
          for (int i = threadIdx.x; i < k; i += blockDim.x) {
            M[(int64_t)col[j] * k + i] = sm[j * k + i];
            V[(int64_t)col[j] * k + i] = sv[j * k + i];
          }
      grid.sync();
    }
    const unsigned long long rot = *(volatile unsigned long long*)&ws[sweep & 1];
    const unsigned long long nbig = *(volatile unsigned long long*)&ws[4 + (sweep & 1)];
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) ws[3] = (unsigned long long)(sweep + 1);
    // converged: no rotation, or only rotations below sqrt(big2) relative, after which the
    // off-diagonal products are O(big2) = O(eps / k) (quadratic convergence), so the next
    // sweep would find nothing above eps
    if (rot == 0 || nbig == 0) break;
  }
}

// sigma_j = |m_j|, U_j = m_j / sigma_j (0 when sigma_j == 0), written in
// descending order of sigma (ties by index): sigma[rank], U[:, rank],
// order[rank] = original column.
__global__ void k_svd_finish(const double* M, int k, double* U, double* sigma, int* order) {
  __shared__ double sig[1024];
  __shared__ double fro2;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0;
    for (int i = 0; i < k; ++i) s = fma(M[(int64_t)j * k + i], M[(int64_t)j * k + i], s);
    sig[j] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0;
    for (int j = 0; j < k; ++j) f = fma(sig[j], sig[j], f);
    fro2 = f;
  }
  __syncthreads();
  // columns at or below the Jacobi negligibility level were never orthogonalised:
  // they get a zero singular vector instead of a normalised rounding residue
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    int rank = 0;
    for (int i = 0; i < k; ++i) rank += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
    order[rank] = j;
    sigma[rank] = sig[j];
    double inv = (sig[j] > 0 && sig[j] * sig[j] > 1e-30 * fro2) ? 1.0 / sig[j] : 0.0;
    for (int i = 0; i < k; ++i) U[(int64_t)rank * k + i] = M[(int64_t)j * k + i] * inv;
  }
}

template <class T, class S>
__global__ void k_convert(const S* in, T* out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)in[e];
}

template <class T>
__global__ void k_sumsq(const T* x, int64_t n, double* out) {
  double s = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double v = (double)x[e];
    s = fma(v, v, s);
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < blockDim.x / 32 ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

__global__ void k_sqrt1(double* x) { x[0] = sqrt(x[0]); }

// out[0] += sum x r, out[1] += sum r r (FP64)
template <class T>
__global__ void k_dot2(const T* x, const T* r, int64_t n, double* out) {
  double a = 0, b = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double xv = (double)x[e], rv = (double)r[e];
    a = fma(xv, rv, a);
    b = fma(rv, rv, b);
  }
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __shared__ double wa[32], wb[32];
  if (threadIdx.x % 32 == 0) {
    wa[threadIdx.x / 32] = a;
    wb[threadIdx.x / 32] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    a = threadIdx.x < blockDim.x / 32 ? wa[threadIdx.x] : 0.0;
    b = threadIdx.x < blockDim.x / 32 ? wb[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (threadIdx.x == 0) {
      atomicAdd(out, a);
      atomicAdd(out + 1, b);
    }
  }
}
// out[0] = out[0] / out[1] (1 when the reference is zero or the ratio is not finite)
__global__ void k_ratio(double* out) {
  const double r = out[1] > 0 ? out[0] / out[1] : 1.0;
  out[0] = (isfinite(r) && r > 0) ? r : 1.0;
}

template <class T>
__global__ void k_scale_inv(T* x, int64_t n, const double* nrm) {
  const double inv = 1.0 / nrm[0];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = (T)((double)x[e] * inv);
}

// dst[c * ld_dst + r] = src[r * ld_src + c] (r < rows, c < cols), zero for
// rows <= r < ld_dst: a padded transpose through 32 x 33 shared tiles.
template <class T>
__global__ void k_transpose_pad(const T* __restrict__ src, int64_t rows, int64_t cols, int64_t ld_src,
                                T* __restrict__ dst, int64_t ld_dst) {
  __shared__ T tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + tx;
    tile[i][tx] = (r < rows && c < cols) ? src[r * ld_src + c] : T(0);
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int64_t c = c0 + i, r = r0 + tx;
    if (c < cols && r < ld_dst) dst[c * ld_dst + r] = tile[tx][i];
  }
}

// dst[c * rows + r] = (T) src[r * cols + c]
template <class T>
__global__ void k_convert_f64_t(const double* __restrict__ src, int64_t rows, int64_t cols, T* __restrict__ dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, r = e % rows;
    dst[e] = (T)src[r * cols + c];
  }
}

template <class T>
__global__ void k_sub(T* out, const T* a, const T* b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = a[e] - b[e];
}

template <class T>
__global__ void k_permute3(const T* in, T* out, int64_t d0, int64_t d1, int64_t d2, int p0, int p1, int p2) {
  // out dims are (d[p0], d[p1], d[p2]); in is [d0][d1][d2]
  const int64_t n = d0 * d1 * d2;
  int64_t d[3] = {d0, d1, d2};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t o2 = e % d[p2], o1 = (e / d[p2]) % d[p1], o0 = e / (d[p2] * d[p1]);
    int64_t idx[3];
    idx[p0] = o0; idx[p1] = o1; idx[p2] = o2;
    out[e] = in[(idx[0] * d1 + idx[1]) * d2 + idx[2]];
  }
}

template <class T>
__global__ void k_fill(T* x, int64_t n, T v) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) x[e] = v;
}

template <class T>
__global__ void k_finite(const T* x, int64_t n, int* flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite((double)x[e])) flag[0] = 1;
}


// ---- small helpers used by the engine -------------------------------------
// s_j = +1 if sum_i w_i X(i, j) >= 0 else -1 (singular-vector sign gauge with
// fixed Gaussian weights w); one block per column
template <class T>
__global__ void k_col_signs(const T* X, int64_t m, int64_t ld, const T* w, double* sgn) {
  const int j = blockIdx.x;
  double s = 0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = fma((double)w[i], (double)X[(int64_t)j * ld + i], s);
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if (threadIdx.x % 32 == 0) ws[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += ws[w];
    sgn[j] = t < 0 ? -1.0 : 1.0;
  }
}

template <class T>
__global__ void k_scale_cols(T* X, int64_t m, int n, int64_t ld, const double* sc) {
  const int64_t tot = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = e / m, i = e % m;
    X[j * ld + i] = (T)((double)X[j * ld + i] * sc[j]);
  }
}

// out(i, j) = X(i, j) * d_j + out(i, j) with d_j = R[j * k + j] (the diagonal of a
// row-major FP64 k x k matrix), one FP32 (or FP64) fused multiply-add per element
template <class T>
__global__ void k_add_diag_cols(const T* X, int64_t m, int n, int64_t ldx, const double* R, int k, T* out,
                                int64_t ldo) {
  const int64_t tot = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / m, i = e % m;
    out[j * ldo + i] = fma(X[j * ldx + i], (T)R[j * (int64_t)k + j], out[j * ldo + i]);
  }
}
template <class T>
__global__ void k_bundle_outer(const T* __restrict__ in, T* __restrict__ out, int64_t rows, int n, int nw) {
  const int B = n * nw * n;
  const int64_t tot = rows * B;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / B;
    const int i = (int)(e % B), xp = i % n, xw = (i / n) % nw, x = i / (n * nw);
    out[r * B + ((int64_t)xw * n + x) * n + xp] = in[e];
  }
}
template <class T>
__global__ void k_zero_diag(T* A, int k, int64_t ld) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) A[j * ld + j] = T(0);
}

__global__ void k_mul_vec(const double* a, const double* b, double* out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] * b[i];
}

__global__ void k_gather_cols(const double* V, const int* order, int k, double* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)k * k; e += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(e / k), i = (int)(e % k);
    out[e] = V[(int64_t)order[r] * k + i];
  }
}

template <class T>
__global__ void k_set_identity(T* X, int64_t m, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = (e / m == e % m) ? T(1) : T(0);
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 152 * 32 ? 152 * 32 : (g < 1 ? 1 : g));
}

}  // namespace

template <class T>
void gaussian_sketch(cudaStream_t s, T* out, int64_t n_rows, int64_t k, int64_t ld, const int64_t* perm_div,
                     uint64_t seed, uint64_t layer, uint64_t w2, uint64_t w3) {
  int64_t hi = perm_div ? perm_div[0] : 1, lo = perm_div ? perm_div[1] : n_rows;
  // algorithmic bytes: the n x k matrix written once (the draws are FP64 arithmetic)
  ProfToken pt = prof_begin(PROF_SKETCH, s, 0.0, (double)sizeof(T) * n_rows * k);
  k_sketch<T><<<grid_for(n_rows * k), 256, 0, s>>>(out, n_rows, k, ld, hi, lo, perm_div ? 1 : 0, seed, layer, w2, w3);
  FP_LAUNCH();
  prof_end(pt, s);
}

template <class T>
void gram_f64(cudaStream_t s, const T* Y, int64_t m, int64_t k, int64_t ld, double* G) {
  FP_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * k * k, s));
  if (sizeof(T) == 4) {
    int tiles = (int)((k + 63) / 64);
    int64_t tri = (int64_t)tiles * (tiles + 1) / 2;
    int64_t nchunk = std::max<int64_t>(1, (152 * 4 + tri - 1) / tri);
    int64_t chunk = ((m + nchunk - 1) / nchunk + 15) / 16 * 16;
    if (chunk < 16) chunk = 16;
    nchunk = (m + chunk - 1) / chunk;
    dim3 grid(tiles, tiles, (unsigned)std::max<int64_t>(nchunk, 1));
    ProfToken pt = prof_begin(PROF_GRAM, s, 2.0 * m * k * k, 4.0 * m * k);
    k_gram_df<<<grid, 256, 0, s>>>((const float*)Y, m, k, ld, chunk, G);
    FP_LAUNCH();
    prof_end(pt, s);
    k_mirror_upper<<<grid_for(k * k), 256, 0, s>>>(G, (int)k);
    FP_LAUNCH();
    return;
  }
  int tiles = (int)((k + 31) / 32);
  int64_t target_blocks = 152 * 8;
  int64_t tri = (int64_t)tiles * (tiles + 1) / 2;
  int64_t nchunk = (target_blocks + tri - 1) / tri;
  int64_t chunk = (m + nchunk - 1) / nchunk;
  chunk = ((chunk + 31) / 32) * 32;
  if (chunk < 32) chunk = 32;
  nchunk = (m + chunk - 1) / chunk;
  if (nchunk < 1) nchunk = 1;
  dim3 grid(tiles, tiles, (unsigned)nchunk);
  ProfToken pt = prof_begin(PROF_GRAM, s, 2.0 * m * k * k, (double)sizeof(T) * m * k);
  k_gram<T><<<grid, 256, 0, s>>>(Y, m, k, ld, chunk, G);
  FP_LAUNCH();
  prof_end(pt, s);
  k_mirror_upper<<<grid_for(k * k), 256, 0, s>>>(G, (int)k);
  FP_LAUNCH();
}

void cholesky_upper_f64(cudaStream_t s, double* G, int k, int* info, double* ws) {
  if (k <= 96) {
    k_cholesky<<<1, 1024, 0, s>>>(G, k, 1e-13, info);
    FP_LAUNCH();
    return;
  }
  static int max_blocks = -1;
  if (max_blocks < 0) {
    int dev = 0, sms = 0, per = 0;
    FP_CUDA(cudaGetDevice(&dev));
    FP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cholesky_coop, 256, 0));
    max_blocks = sms * std::max(per, 0);
  }
  int blocks = std::min(max_blocks, 152);
  FP_CHECK(blocks >= 1, FPEPS_ERR_CUDA, "cholesky: no co-resident blocks");
  double tol = 1e-13;
  void* args[] = {&G, &k, &tol, &info, &ws};
  ProfToken pt = prof_begin(PROF_FACTOR, s, (double)k * k * k / 3.0, 8.0 * k * k);
  count_launch();
  FP_CUDA(cudaLaunchCooperativeKernel((void*)k_cholesky_coop, blocks, 256, args, 0, s));
  prof_end(pt, s);
}

void tri_inverse_upper_f64(cudaStream_t s, const double* R, int k, double* Rinv) {
  const int wpb = 4;
  size_t smem = (size_t)wpb * k * sizeof(double);
  static bool attr = false;
  if (!attr) {
    FP_CUDA(cudaFuncSetAttribute(k_tri_inverse_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 1024 * 8));
    attr = true;
  }
  FP_CHECK(k <= 1024, FPEPS_ERR_UNSUPPORTED, "tri_inverse: k > 1024");
  k_tri_inverse_warp<<<(k + wpb - 1) / wpb, wpb * 32, smem, s>>>(R, k, Rinv);
  FP_LAUNCH();
}

void svd_jacobi_f64(cudaStream_t s, double* Mat, int k, double* U, double* sigma, double* V, int* order, int* info,
                    void* ws_dev) {
  FP_CHECK(k <= 1024, FPEPS_ERR_UNSUPPORTED, "svd: k > 1024");
  if (k <= 96) {
    // stopping rule |m_p.m_q| <= sqrt(k) eps |m_p||m_q|: a dot product of length k
    // carries rounding of that size, so a fixed 1e-15 could never be met
    k_jacobi_svd<<<1, 1024, 0, s>>>(Mat, V, k, 30, 1e-15 * sqrt((double)k), info);
    FP_LAUNCH();
  } else {
    // one CTA per pair of two-column blocks, all co-resident (cooperative launch)
    const int nb = (k + 1) / 2, blocks = (nb + (nb & 1)) / 2;
    const size_t smem = (8 * (size_t)k + 12) * sizeof(double);
    static bool attr = false;
    static int max_blocks = -1;
    if (!attr) {
      FP_CUDA(cudaFuncSetAttribute(k_jacobi_svd_blk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)((8 * 1024 + 12) * sizeof(double))));
      int dev = 0, sms = 0, per = 0;
      FP_CUDA(cudaGetDevice(&dev));
      FP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_jacobi_svd_blk, JB_THREADS,
                                                            (8 * 1024 + 12) * sizeof(double)));
      max_blocks = sms * std::max(per, 0);
      attr = true;
    }
    FP_CHECK(blocks <= max_blocks, FPEPS_ERR_CUDA, "svd: too few co-resident blocks");
    void* fn = (void*)k_jacobi_svd_blk;
    unsigned long long* ws = (unsigned long long*)ws_dev;
    int max_sweeps = 30;
    double eps = 1e-15 * sqrt((double)k);
    double big2 = eps / k;
    void* args[] = {&Mat, &V, &k, &max_sweeps, &eps, &big2, &ws};
    ProfToken pt = prof_begin(PROF_FACTOR, s, 0.0, 16.0 * k * k);
    count_launch();
    FP_CUDA(cudaLaunchCooperativeKernel(fn, blocks, JB_THREADS, args, smem, s));
    prof_end(pt, s);
    FP_CUDA(cudaMemsetAsync(info, 0, sizeof(int), s));
    static const bool trace = getenv("FPEPS_TRACE_SVD") != nullptr;   // diagnostics: sweeps used
    if (trace) {
      unsigned long long sw = 0;
      FP_CUDA(cudaMemcpyAsync(&sw, ws + 3, sizeof(sw), cudaMemcpyDeviceToHost, s));
      FP_CUDA(cudaStreamSynchronize(s));
      fprintf(stderr, "[fpeps] jacobi k=%d sweeps=%llu\n", k, sw);
    }
  }
  k_svd_finish<<<1, 1024, 0, s>>>(Mat, k, U, sigma, order);
  FP_LAUNCH();
}

template <class T>
void convert_f64(cudaStream_t s, const double* in, T* out, int64_t n) {
  k_convert<T, double><<<grid_for(n), 256, 0, s>>>(in, out, n);
  FP_LAUNCH();
}
template <class T>
void to_f64(cudaStream_t s, const T* in, double* out, int64_t n) {
  k_convert<double, T><<<grid_for(n), 256, 0, s>>>(in, out, n);
  FP_LAUNCH();
}

template <class T>
void frob_norm_f64(cudaStream_t s, const T* x, int64_t n, double* out) {
  FP_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  k_sumsq<T><<<grid_for(n), 256, 0, s>>>(x, n, out);
  FP_LAUNCH();
  k_sqrt1<<<1, 1, 0, s>>>(out);
  FP_LAUNCH();
}

template <class T>
void scale_against(cudaStream_t s, const T* x, const T* r, int64_t n, double* out) {
  FP_CUDA(cudaMemsetAsync(out, 0, 2 * sizeof(double), s));
  k_dot2<T><<<grid_for(n), 256, 0, s>>>(x, r, n, out);
  FP_LAUNCH();
  k_ratio<<<1, 1, 0, s>>>(out);
  FP_LAUNCH();
}

template <class T>
void scale_by_inv(cudaStream_t s, T* x, int64_t n, const double* nrm) {
  k_scale_inv<T><<<grid_for(n), 256, 0, s>>>(x, n, nrm);
  FP_LAUNCH();
}

template <class T>
void sub_into(cudaStream_t s, T* out, const T* a, const T* b, int64_t n) {
  if (n <= 0) return;
  k_sub<T><<<grid_for(n), 256, 0, s>>>(out, a, b, n);
  FP_LAUNCH();
}

template <class T>
void transpose_pad(cudaStream_t s, const T* src, int64_t rows, int64_t cols, int64_t ld_src, T* dst, int64_t ld_dst) {
  if (rows <= 0 || cols <= 0) return;
  const int64_t gy = (ld_dst + 31) / 32, gx = (cols + 31) / 32;
  FP_CHECK(gy < 65536, FPEPS_ERR_UNSUPPORTED, "transpose: too many rows");
  k_transpose_pad<T><<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, s>>>(src, rows, cols, ld_src, dst, ld_dst);
  FP_LAUNCH();
}

template <class T>
void add_diag_cols(cudaStream_t s, const T* X, int64_t m, int n, int64_t ldx, const double* R, int k, T* out,
                   int64_t ldo) {
  if (m * n == 0) return;
  k_add_diag_cols<T><<<grid_for(m * n), 256, 0, s>>>(X, m, n, ldx, R, k, out, ldo);
  FP_LAUNCH();
}
template <class T>
void bundle_outer(cudaStream_t s, const T* in, T* out, int64_t rows, int n, int nw) {
  const int64_t tot = rows * n * nw * n;
  if (tot == 0) return;
  k_bundle_outer<T><<<grid_for(tot), 256, 0, s>>>(in, out, rows, n, nw);
  FP_LAUNCH();
}
template <class T>
void zero_diag(cudaStream_t s, T* A, int k, int64_t ld) {
  if (k <= 0) return;
  k_zero_diag<T><<<(k + 255) / 256, 256, 0, s>>>(A, k, ld);
  FP_LAUNCH();
}

template <class T>
void convert_f64_t(cudaStream_t s, const double* src, int64_t rows, int64_t cols, T* dst) {
  k_convert_f64_t<T><<<grid_for(rows * cols), 256, 0, s>>>(src, rows, cols, dst);
  FP_LAUNCH();
}

template <class T>
void permute3(cudaStream_t s, const T* in, T* out, int64_t d0, int64_t d1, int64_t d2, int p0, int p1, int p2) {
  k_permute3<T><<<grid_for(d0 * d1 * d2), 256, 0, s>>>(in, out, d0, d1, d2, p0, p1, p2);
  FP_LAUNCH();
}

template <class T>
void fill(cudaStream_t s, T* x, int64_t n, T v) {
  if (n <= 0) return;
  k_fill<T><<<grid_for(n), 256, 0, s>>>(x, n, v);
  FP_LAUNCH();
}

template <class T>
void check_finite(cudaStream_t s, const T* x, int64_t n, int* flag) {
  if (n <= 0) return;
  k_finite<T><<<grid_for(n), 256, 0, s>>>(x, n, flag);
  FP_LAUNCH();
}


template <class T>
void col_signs(cudaStream_t s, const T* X, int64_t m, int n, int64_t ld, const T* w, double* sgn) {
  if (n <= 0) return;
  k_col_signs<T><<<n, 256, 0, s>>>(X, m, ld, w, sgn);
  FP_LAUNCH();
}
template <class T>
void scale_cols(cudaStream_t s, T* X, int64_t m, int n, int64_t ld, const double* sc) {
  if (n <= 0 || m <= 0) return;
  k_scale_cols<T><<<grid_for(m * n), 256, 0, s>>>(X, m, n, ld, sc);
  FP_LAUNCH();
}
void mul_vec(cudaStream_t s, const double* a, const double* b, double* out, int n) {
  k_mul_vec<<<(n + 255) / 256, 256, 0, s>>>(a, b, out, n);
  FP_LAUNCH();
}
void gather_cols_f64(cudaStream_t s, const double* V, const int* order, int k, double* out) {
  k_gather_cols<<<grid_for((int64_t)k * k), 256, 0, s>>>(V, order, k, out);
  FP_LAUNCH();
}
template <class T>
void set_identity(cudaStream_t s, T* X, int64_t m, int n) {
  k_set_identity<T><<<grid_for(m * n), 256, 0, s>>>(X, m, n);
  FP_LAUNCH();
}
template <class T>
void copy_cols(cudaStream_t s, const T* src, int64_t m, int n, T* dst) {
  FP_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * m * n, cudaMemcpyDeviceToDevice, s));
}

// Row selection within every column of a column-major block (charge sectors of
// the block-sparse mode): gather dst[i + j ldd] = src[idx[i] + j lds], scatter
// dst[idx[i] + j ldd] = src[i + j lds], for i < n, j < k. idx holds valid rows of
// the indexed side (checked on the host when the lists are built).
template <class T>
__global__ void k_gather_rows(const T* __restrict__ src, int64_t lds, const int64_t* __restrict__ idx, int64_t n,
                              int64_t k, T* __restrict__ dst, int64_t ldd) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e % n;
    dst[j * ldd + i] = src[j * lds + idx[i]];
  }
}
template <class T>
__global__ void k_scatter_rows(const T* __restrict__ src, int64_t lds, const int64_t* __restrict__ idx, int64_t n,
                               int64_t k, T* __restrict__ dst, int64_t ldd) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, i = e % n;
    dst[j * ldd + idx[i]] = src[j * lds + i];
  }
}
template <class T>
void gather_rows(cudaStream_t s, const T* src, int64_t lds, const int64_t* idx, int64_t n, int64_t k, T* dst,
                 int64_t ldd) {
  if (n * k == 0) return;
  k_gather_rows<T><<<grid_for(n * k), 256, 0, s>>>(src, lds, idx, n, k, dst, ldd);
  FP_LAUNCH();
}
template <class T>
void scatter_rows(cudaStream_t s, const T* src, int64_t lds, const int64_t* idx, int64_t n, int64_t k, T* dst,
                  int64_t ldd) {
  if (n * k == 0) return;
  k_scatter_rows<T><<<grid_for(n * k), 256, 0, s>>>(src, lds, idx, n, k, dst, ldd);
  FP_LAUNCH();
}

// dst (cols x rows, column-major, ld ldd) = transpose of src (rows x cols, ld lds)
template <class T>
__global__ void k_transpose_block(const T* __restrict__ src, int64_t lds, int64_t rows, int64_t cols,
                                  T* __restrict__ dst, int64_t ldd) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / rows, i = e % rows;
    dst[i * ldd + j] = src[j * lds + i];
  }
}
template <class T>
void transpose_block(cudaStream_t s, const T* src, int64_t lds, int64_t rows, int64_t cols, T* dst, int64_t ldd) {
  if (rows * cols == 0) return;
  k_transpose_block<T><<<grid_for(rows * cols), 256, 0, s>>>(src, lds, rows, cols, dst, ldd);
  FP_LAUNCH();
}

#define INST(T)                                                                                              \
  template void gaussian_sketch<T>(cudaStream_t, T*, int64_t, int64_t, int64_t, const int64_t*, uint64_t,    \
                                   uint64_t, uint64_t, uint64_t);                                            \
  template void gram_f64<T>(cudaStream_t, const T*, int64_t, int64_t, int64_t, double*);                      \
  template void convert_f64<T>(cudaStream_t, const double*, T*, int64_t);                                    \
  template void to_f64<T>(cudaStream_t, const T*, double*, int64_t);                                          \
  template void frob_norm_f64<T>(cudaStream_t, const T*, int64_t, double*);                                  \
  template void scale_by_inv<T>(cudaStream_t, T*, int64_t, const double*);                                   \
  template void scale_against<T>(cudaStream_t, const T*, const T*, int64_t, double*);                        \
  template void permute3<T>(cudaStream_t, const T*, T*, int64_t, int64_t, int64_t, int, int, int);            \
  template void transpose_pad<T>(cudaStream_t, const T*, int64_t, int64_t, int64_t, T*, int64_t);            \
  template void sub_into<T>(cudaStream_t, T*, const T*, const T*, int64_t);                                   \
  template void convert_f64_t<T>(cudaStream_t, const double*, int64_t, int64_t, T*);                         \
  template void add_diag_cols<T>(cudaStream_t, const T*, int64_t, int, int64_t, const double*, int, T*, int64_t); \
  template void zero_diag<T>(cudaStream_t, T*, int, int64_t);                                                 \
  template void bundle_outer<T>(cudaStream_t, const T*, T*, int64_t, int, int);                               \
  template void fill<T>(cudaStream_t, T*, int64_t, T);                                                        \
  template void check_finite<T>(cudaStream_t, const T*, int64_t, int*);                                      \
  template void col_signs<T>(cudaStream_t, const T*, int64_t, int, int64_t, const T*, double*);                         \
  template void scale_cols<T>(cudaStream_t, T*, int64_t, int, int64_t, const double*);                        \
  template void set_identity<T>(cudaStream_t, T*, int64_t, int);                                              \
  template void copy_cols<T>(cudaStream_t, const T*, int64_t, int, T*);                                      \
  template void gather_rows<T>(cudaStream_t, const T*, int64_t, const int64_t*, int64_t, int64_t, T*, int64_t);   \
  template void scatter_rows<T>(cudaStream_t, const T*, int64_t, const int64_t*, int64_t, int64_t, T*, int64_t); \
  template void transpose_block<T>(cudaStream_t, const T*, int64_t, int64_t, int64_t, T*, int64_t);
INST(float)
INST(double)
template void fill<int>(cudaStream_t, int*, int64_t, int);

}  // namespace fpeps
