// Internal declarations shared by the CUDA translation units of libfpeps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fpeps.h"

namespace fpeps {

// ---------------------------------------------------------------- errors
struct Error {
  fpeps_status st;
  std::string msg;
};

#define FP_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::fpeps::Error{FPEPS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define FP_CHECK(cond, code, text)                                   \
  do {                                                               \
    if (!(cond)) throw ::fpeps::Error{code, std::string(text)};      \
  } while (0)

// ---------------------------------------------------------------- launch accounting
// Every kernel launch of the library goes through FP_LAUNCH (count), and the
// hot kernel classes can be bracketed with CUDA events (prof_begin/prof_end)
// when profiling is enabled, so callers can time them on their own stream.
enum ProfKind {
  PROF_GEMM_TC = 0, PROF_GEMM_SIMT = 1, PROF_SANDWICH = 2, PROF_GRAM = 3, PROF_FACTOR = 4, PROF_SKETCH = 5, PROF_KINDS = 6
};
void count_launch();
struct ProfToken {
  int kind = -1;
  cudaEvent_t e0 = nullptr;
  double flops = 0, bytes = 0;
};
ProfToken prof_begin(int kind, cudaStream_t s, double flops, double bytes);
void prof_end(ProfToken& t, cudaStream_t s);

#define FP_LAUNCH()                  \
  do {                               \
    ::fpeps::count_launch();         \
    FP_CUDA(cudaGetLastError());     \
  } while (0)

// ---------------------------------------------------------------- memory
// Device memory owned through the env allocator. Arena buffers are released in
// bulk when the arena is reset.
struct Allocator {
  fpeps_allocator a{};
  bool has = false;
  cudaStream_t stream = nullptr;
  void* get(size_t bytes);
  void put(void* p);
};

struct Arena {
  Allocator* al = nullptr;
  std::vector<void*> live;
  void* get(size_t bytes) {
    void* p = al->get(bytes < 256 ? 256 : bytes);
    live.push_back(p);
    return p;
  }
  template <class T>
  T* get_n(size_t n) { return static_cast<T*>(get(n * sizeof(T))); }
  void reset() {
    for (void* p : live) al->put(p);
    live.clear();
  }
  ~Arena() { reset(); }
};

// ---------------------------------------------------------------- GEMM
// C(m,n) = alpha * sum_k A(m,k) B(n,k) + beta * C(m,n)
//   A(m,k) = A[m*a_m + k*a_k], B(n,k) = B[n*b_n + k*b_k]
//   addr(C(m,n)) = (m/mdiv)*c0 + (m%mdiv)*c1 + (n/ndiv)*c2 + (n%ndiv)*c3
struct OutMap {
  int64_t mdiv, c0, c1, ndiv, c2, c3;
};
inline OutMap out_rowmajor(int64_t M, int64_t N, int64_t ldc) { return OutMap{M, 0, ldc, N, 0, 1}; }
inline OutMap out_colmajor(int64_t M, int64_t N, int64_t ldc) { return OutMap{M, 0, 1, N, 0, ldc}; }

template <class T>
void gemm_simt(cudaStream_t s, int64_t M, int64_t N, int64_t K, T alpha, const T* A, int64_t a_m,
               int64_t a_k, const T* B, int64_t b_n, int64_t b_k, T beta, T* C, OutMap om);

// Tensor-core GEMM for K-major A [M][lda] and B [N][ldb] (k contiguous), split
// precision (mode 2 = 3xTF32, 3 = 3xBF16). Returns false if the shape is not
// supported by the tensor-core path (caller falls back to nothing: it is an error).
bool gemm_tc_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb);
void gemm_tc(cudaStream_t s, int mode, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
             const float* B, int64_t ldb, float* C, OutMap om, void* scratch, size_t scratch_bytes,
             bool hold_loads = false);   // hold_loads: self-test of the bounded waits (no loads issued)
size_t gemm_tc_scratch_bytes(int mode, int64_t M, int64_t N, int64_t K);

// ---------------------------------------------------------------- sandwich
// Bundle order. A (ket, PEPO, bra) bundle of dims (n, nw, n) is indexed (x nw + x_w) n + x'
// everywhere except in the output of the sandwich, where the output bundle with unit stride
// (the one the next GEMM contracts over) is stored PEPO-index outermost, (x_w n + x) n + x':
// one output pair (v_w, z_w) then owns contiguous runs of n^2 elements. The operand that
// the next GEMM contracts with that bundle is stored in the same order (bundle_outer).
__host__ __device__ inline int64_t bundle_index(int x, int xw, int xp, int n, int nw, bool pepo_outer) {
  return pepo_outer ? ((int64_t)xw * n + x) * n + xp : ((int64_t)x * nw + xw) * n + xp;
}
// out[r][(x_w n + x) n + x'] = in[r][(x nw + x_w) n + x'] for r < rows
template <class T>
void bundle_outer(cudaStream_t s, const T* in, T* out, int64_t rows, int n, int nw);

// One orientation of the site sandwich: inputs legs (x, y) -> outputs (v, z).
struct SandOrient {
  int nx, nxw, ny, nyw, nv, nvw, nz, nzw, p;
  int nch;                 // nonzero PEPO channels
  const int* d_ch;         // [nch][4] = (xw, yw, vw, zw), sorted by (vw, zw)
  const int* d_pair_off;   // [nvw*nzw + 1] channel offsets per (vw, zw)
  const void* d_aw;        // [nch][nx][ny][nv][nz][p']  (A . W_ch)
  const void* d_ar;        // [nx][ny][nv][nz][p]        (A in these roles)
  int ch_host_max_per_pair;
  // tcgen05 sandwich (FP32 data): hi/lo operand images of A . W_ch and of the bra
  const void* d_kimg = nullptr;
  const void* d_arimg = nullptr;
};

template <class T>
void sandwich_apply(cudaStream_t s, const SandOrient& o, int64_t nt, int64_t nk, const T* in,
                    int64_t i_t, int64_t i_k, int64_t i_X, int64_t i_Y, T* out, int64_t o_t, int64_t o_k,
                    int64_t o_V, int64_t o_Z);

// 3xTF32 tensor-core version (mma.sync), float data; needs D <= 6 and D^2 p <= 144.
bool sandwich_mma_fits(const SandOrient& o);
void sandwich_apply_tc(cudaStream_t s, const SandOrient& o, int64_t nt, int64_t nk, const float* in, int64_t i_t,
                       int64_t i_k, int64_t i_X, int64_t i_Y, float* out, int64_t o_t, int64_t o_k, int64_t o_V,
                       int64_t o_Z);

// tcgen05 3xTF32 version (sandwich_tc.cu), float data; needs D <= 6, p <= 4 and p D^2 <= 144.
// The operand images are built once per site and orientation (sandwich_tc_images, sizes from
// sandwich_tc_image_floats); err is the tensor-core error word (set to 1 when a bounded wait
// timed out).
bool sandwich_tc_fits(const SandOrient& o);
void sandwich_tc_image_floats(const SandOrient& o, size_t* ket, size_t* bra);
void sandwich_tc_images(cudaStream_t s, const SandOrient& o, float* ket_img, float* bra_img);
void sandwich_apply_tcgen05(cudaStream_t s, const SandOrient& o, int64_t nt, int64_t nk, const float* in,
                            int64_t i_t, int64_t i_k, int64_t i_X, int64_t i_Y, float* out, int64_t o_t, int64_t o_k,
                            int64_t o_V, int64_t o_Z, int* err);

// Builds the role-permuted ket and the channel products A.W_ch for one orientation.
// roles[4] = leg index (0..3 = l,u,r,d) of (x, y, v, z).
template <class T>
void sandwich_prepare(cudaStream_t s, const T* A, const int dA[5], const T* W, const int dW[6], const int roles[4],
                      const int* d_ch, int nch, T* d_aw, T* d_ar);

// PEPO channel scan: flags[l,u,r,d] = 1 if block W[l,u,r,d,:,:] has a nonzero.
template <class T>
void pepo_scan(cudaStream_t s, const T* W, const int dW[6], int* d_flags);

// Row-0 boundary T[L][Dn][R] from the sandwich with the dimension-1 up legs.
template <class T>
void first_row_tensor(cudaStream_t s, const T* A, const int dA[5], const T* W, const int dW[6], T* out);

// ---------------------------------------------------------------- linalg
template <class T>
void gaussian_sketch(cudaStream_t s, T* out, int64_t n_rows, int64_t k, int64_t ld, const int64_t* perm_div,
                     uint64_t seed, uint64_t layer, uint64_t w2, uint64_t w3);

template <class T>
void gram_f64(cudaStream_t s, const T* Y, int64_t m, int64_t k, int64_t ld, double* G);

// returns device status word pointer semantics: info[0] != 0 on failure
// ws: >= 8 bytes of device scratch
void cholesky_upper_f64(cudaStream_t s, double* G, int k, int* info, double* ws);
void tri_inverse_upper_f64(cudaStream_t s, const double* R, int k, double* Rinv);
void sym_eig_jacobi_f64(cudaStream_t s, double* G, int k, double* evec, double* eval, int* info);
// One-sided Jacobi SVD of the k x k col-major Mat (destroyed): Mat = U diag(sigma) V^T,
// sigma descending; U columns sorted, V columns in original order with order[rank] =
// original column. ws_dev: >= 64 bytes of device scratch.
void svd_jacobi_f64(cudaStream_t s, double* Mat, int k, double* U, double* sigma, double* V, int* order,
                    int* info, void* ws_dev);

void gather_cols_f64(cudaStream_t s, const double* V, const int* order, int k, double* out);

template <class T>
void convert_f64(cudaStream_t s, const double* in, T* out, int64_t n);
template <class T>
void to_f64(cudaStream_t s, const T* in, double* out, int64_t n);

template <class T>
void frob_norm_f64(cudaStream_t s, const T* x, int64_t n, double* out);
template <class T>
void scale_by_inv(cudaStream_t s, T* x, int64_t n, const double* nrm);
// out[0] = <x, r> / <r, r> in FP64 (1 if that is not a positive finite number);
// out: >= 2 doubles of device memory
template <class T>
void scale_against(cudaStream_t s, const T* x, const T* r, int64_t n, double* out);

template <class T>
void permute3(cudaStream_t s, const T* in, T* out, int64_t d0, int64_t d1, int64_t d2, int p0, int p1, int p2);
// dst[c * ld_dst + r] = src[r * ld_src + c] for r < rows, c < cols; zero for rows <= r < ld_dst
template <class T>
void transpose_pad(cudaStream_t s, const T* src, int64_t rows, int64_t cols, int64_t ld_src, T* dst, int64_t ld_dst);
// out = a - b elementwise (out may alias a or b)
template <class T>
void sub_into(cudaStream_t s, T* out, const T* a, const T* b, int64_t n);
// out(i, j) += X(i, j) * R[j * k + j] for i < m, j < n (X, out column-major; R row-major FP64 k x k)
template <class T>
void add_diag_cols(cudaStream_t s, const T* X, int64_t m, int n, int64_t ldx, const double* R, int k, T* out,
                   int64_t ldo);
// A[j * ld + j] = 0 for j < k
template <class T>
void zero_diag(cudaStream_t s, T* A, int k, int64_t ld);
// dst (col-major rows x cols) = (T) src (row-major rows x cols)
template <class T>
void convert_f64_t(cudaStream_t s, const double* src, int64_t rows, int64_t cols, T* dst);

template <class T>
void fill(cudaStream_t s, T* x, int64_t n, T v);

template <class T>
void check_finite(cudaStream_t s, const T* x, int64_t n, int* flag);

}  // namespace fpeps
