// CUDA-core GEMMs with arbitrary operand strides and a split-index output map.
//
// This is the FP64 path and the plain-FP32 path of every contraction of the
// Fig. 2(a) pattern (boundary x vectors, environment x vectors), and the
// general small-matrix product of the rSVD steps (projections, Q = Y R^-1).
//   C(m,n) = alpha * sum_k A(m,k) B(n,k) + beta * C(m,n)
#include "common.cuh"

namespace fpeps {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;   // 256 threads, 4x4 per thread

template <class T>
__global__ void __launch_bounds__(256) k_gemm(int64_t M, int64_t N, int64_t K, T alpha, const T* __restrict__ A,
                                              int64_t a_m, int64_t a_k, const T* __restrict__ B, int64_t b_n,
                                              int64_t b_k, T beta, T* __restrict__ C, OutMap om) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int tr = tid / 16, tc = tid % 16;   // 16 x 16 thread grid
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  // load mapping: if k is the contiguous axis, consecutive threads walk k
  const bool a_kfast = (a_k == 1);
  const bool b_kfast = (b_k == 1);
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int mm, kk;
      if (a_kfast) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[gm * a_m + gk * a_k] : T(0);
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int nn, kk;
      if (b_kfast) { nn = e / BK; kk = e % BK; } else { kk = e / BN; nn = e % BN; }
      int64_t gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? B[gn * b_n + gk * b_k] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int64_t gm = m0 + tr + 16 * i;
    if (gm >= M) continue;
    int64_t mo = (gm / om.mdiv) * om.c0 + (gm % om.mdiv) * om.c1;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t gn = n0 + tc + 16 * j;
      if (gn >= N) continue;
      int64_t addr = mo + (gn / om.ndiv) * om.c2 + (gn % om.ndiv) * om.c3;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v += beta * C[addr];
      C[addr] = v;
    }
  }
}

// FP32 products with at least one 128 x 128 output tile: 256 threads, 8 x 8 outputs per
// thread (two 4-wide strips in each direction, so the shared-memory reads are float4 and
// conflict-free), k-tiles of 8 double-buffered in shared memory with the next tile's loads
// held in registers while the current one is used. MF: the thread index runs along m first
// (column-major outputs store 64 contiguous floats per warp row), else along n.
constexpr int GB = 128, GK = 8;
template <bool MF>
__global__ void __launch_bounds__(256) k_gemm_big(int64_t M, int64_t N, int64_t K, float alpha,
                                                  const float* __restrict__ A, int64_t a_m, int64_t a_k,
                                                  const float* __restrict__ B, int64_t b_n, int64_t b_k, float beta,
                                                  float* __restrict__ C, OutMap om) {
  __shared__ __align__(16) float As[2][GK][GB + 4];
  __shared__ __align__(16) float Bs[2][GK][GB + 4];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.y * GB, n0 = (int64_t)blockIdx.x * GB;
  const int tf = tid % 16, ts = tid / 16;
  const int tm = MF ? tf : ts, tn = MF ? ts : tf;   // 4-wide strips at 4 tm, 64 + 4 tm (and for n)
  // loads: 4 elements of A and 4 of B per thread per k-tile, along the operand's contiguous axis
  const bool akf = a_k == 1, bkf = b_k == 1;
  float ra[4], rb[4];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      const int mm = akf ? e / GK : e % GB, kk = akf ? e % GK : e / GB;
      const int64_t gm = m0 + mm, gk = k0 + kk;
      ra[u] = (gm < M && gk < K) ? A[gm * a_m + gk * a_k] : 0.f;
      const int nn = bkf ? e / GK : e % GB, kb = bkf ? e % GK : e / GB;
      const int64_t gn = n0 + nn, gkb = k0 + kb;
      rb[u] = (gn < N && gkb < K) ? B[gn * b_n + gkb * b_k] : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      const int mm = akf ? e / GK : e % GB, kk = akf ? e % GK : e / GB;
      As[buf][kk][mm] = ra[u];
      const int nn = bkf ? e / GK : e % GB, kb = bkf ? e % GK : e / GB;
      Bs[buf][kb][nn] = rb[u];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int64_t k0 = 0; k0 < K; k0 += GK) {
    const bool more = k0 + GK < K;
    if (more) load(k0 + GK);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a0 = *(const float4*)&As[buf][kk][4 * tm], a1 = *(const float4*)&As[buf][kk][64 + 4 * tm];
      const float4 b0 = *(const float4*)&Bs[buf][kk][4 * tn], b1 = *(const float4*)&Bs[buf][kk][64 + 4 * tn];
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = m0 + (i < 4 ? 4 * tm + i : 64 + 4 * tm + i - 4);
    if (gm >= M) continue;
    const int64_t mo = (gm / om.mdiv) * om.c0 + (gm % om.mdiv) * om.c1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t gn = n0 + (j < 4 ? 4 * tn + j : 64 + 4 * tn + j - 4);
      if (gn >= N) continue;
      const int64_t addr = mo + (gn / om.ndiv) * om.c2 + (gn % om.ndiv) * om.c3;
      float v = alpha * acc[i][j];
      if (beta != 0.f) v += beta * C[addr];
      C[addr] = v;
    }
  }
}

}  // namespace

template <class T>
void gemm_simt(cudaStream_t s, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t a_m, int64_t a_k,
               const T* B, int64_t b_n, int64_t b_k, T beta, T* C, OutMap om) {
  if (M <= 0 || N <= 0) return;
  FP_CHECK(om.mdiv > 0 && om.ndiv > 0, FPEPS_ERR_ARG, "gemm: bad output map");
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  FP_CHECK(grid.y <= 65535u, FPEPS_ERR_UNSUPPORTED, "gemm: M too large for grid");
  ProfToken pt = prof_begin(PROF_GEMM_SIMT, s, 2.0 * M * N * K,
                            (double)sizeof(T) * ((double)M * K + (double)N * K + (double)M * N));
  if (sizeof(T) == 4 && M >= GB && N >= GB) {
    dim3 g2((unsigned)((N + GB - 1) / GB), (unsigned)((M + GB - 1) / GB));
    FP_CHECK(g2.y <= 65535u, FPEPS_ERR_UNSUPPORTED, "gemm: M too large for grid");
    if (om.c1 == 1)
      k_gemm_big<true><<<g2, 256, 0, s>>>(M, N, K, (float)alpha, (const float*)A, a_m, a_k, (const float*)B, b_n, b_k,
                                          (float)beta, (float*)C, om);
    else
      k_gemm_big<false><<<g2, 256, 0, s>>>(M, N, K, (float)alpha, (const float*)A, a_m, a_k, (const float*)B, b_n,
                                           b_k, (float)beta, (float*)C, om);
  } else {
    k_gemm<T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, a_m, a_k, B, b_n, b_k, beta, C, om);
  }
  FP_LAUNCH();
  prof_end(pt, s);
}

template void gemm_simt<float>(cudaStream_t, int64_t, int64_t, int64_t, float, const float*, int64_t, int64_t,
                               const float*, int64_t, int64_t, float, float*, OutMap);
template void gemm_simt<double>(cudaStream_t, int64_t, int64_t, int64_t, double, const double*, int64_t, int64_t,
                                const double*, int64_t, int64_t, double, double*, OutMap);

}  // namespace fpeps
