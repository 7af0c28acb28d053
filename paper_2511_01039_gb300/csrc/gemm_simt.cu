// CUDA-core GEMM with arbitrary operand strides and a split-index output map.
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
  k_gemm<T><<<grid, 256, 0, s>>>(M, N, K, alpha, A, a_m, a_k, B, b_n, b_k, beta, C, om);
  FP_LAUNCH();
  prof_end(pt, s);
}

template void gemm_simt<float>(cudaStream_t, int64_t, int64_t, int64_t, float, const float*, int64_t, int64_t,
                               const float*, int64_t, int64_t, float, float*, OutMap);
template void gemm_simt<double>(cudaStream_t, int64_t, int64_t, int64_t, double, const double*, int64_t, int64_t,
                                const double*, int64_t, int64_t, double, double*, OutMap);

}  // namespace fpeps
