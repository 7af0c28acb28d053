// Row engine: boundary initialisation, zip-up rSVD compression, CBE fit and
// the exact closing of the last row (paper Sec. II and Sec. IV).
//
// Layouts (device, compute precision T):
//   boundary  T_c   [t][U][t']            (plus per-site copies [t'][t][U],
//                                          [t][t'][U], [t'][U][t] for the GEMMs)
//   left env  EL_c  [a][t][L]   and [t][L][a]
//   right env ER_c  [a][t'][R]  and [t'][R][a]
//   blocks of k vectors: [k][bundle][bond]  (bond fastest), e.g. X [k][R][t'],
//   Y [k][Dn][a]; in C order of the (bond, bundle) legs the flat index of such
//   a vector element is bond * |bundle| + bundle (this is the sketch counter).
// Every contraction is a "TN" GEMM C(m,n) = sum_k A[m][k] B[n][k] with both
// operands k-contiguous (Fig. 2(a) pattern: boundary x vectors, sandwich,
// environment x vectors), sliced over the k vectors so that the O(chi^2 (DwD)^2)
// intermediates of Sec. III never exist in full.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <functional>
#include <map>

#include "env.cuh"

namespace fpeps {

template <class T>
void col_signs(cudaStream_t s, const T* X, int64_t m, int n, int64_t ld, const T* w, double* sgn);
template <class T>
void scale_cols(cudaStream_t s, T* X, int64_t m, int n, int64_t ld, const double* colscale);
void mul_vec(cudaStream_t s, const double* a, const double* b, double* out, int n);
void gather_cols_f64(cudaStream_t s, const double* V, const int* order, int k, double* out);
template <class T>
void set_identity(cudaStream_t s, T* X, int64_t m, int n);
template <class T>
void copy_cols(cudaStream_t s, const T* src, int64_t m, int n, T* dst);
template <class T>
void gather_rows(cudaStream_t s, const T* src, int64_t lds, const int64_t* idx, int64_t n, int64_t k, T* dst,
                 int64_t ldd);
template <class T>
void scatter_rows(cudaStream_t s, const T* src, int64_t lds, const int64_t* idx, int64_t n, int64_t k, T* dst,
                  int64_t ldd);
template <class T>
void transpose_block(cudaStream_t s, const T* src, int64_t lds, int64_t rows, int64_t cols, T* dst, int64_t ldd);

namespace {

enum Orient { FWD = 0, BWD = 1, RF = 2, RB = 3 };
const int kRoles[4][4] = {{1, 2, 0, 3}, {0, 3, 1, 2}, {2, 3, 0, 1}, {0, 1, 2, 3}};

inline int bund(const SiteHost& h, int leg) { return h.dA[leg] * h.dW[leg] * h.dA[leg]; }

}  // namespace

// ------------------------------------------------------------------ sandwich data
void ensure_sandwich(fpeps_env* env, int layer, int row) {
  const int Ly = env->cfg.Ly;
  auto& sv = env->sand[layer];
  if (sv.empty()) sv.resize((size_t)env->cfg.Lx * Ly);
  for (int c = 0; c < Ly; ++c) {
    const int idx = row * Ly + c;
    SiteSand& sd = sv[idx];
    if (!sd.bufs.empty()) continue;
    const SiteHost& h = env->sites[layer][idx];
    const int nch = (int)h.ch.size() / 4;
    const int p = h.dA[4];
    for (int o = 0; o < 4; ++o) {
      const int* ro = kRoles[o];
      // channels in role order, sorted by (v_w, z_w)
      std::vector<std::array<int, 4>> rc;
      for (int i = 0; i < nch; ++i) {
        const int* v = &h.ch[4 * i];
        rc.push_back({v[ro[0]], v[ro[1]], v[ro[2]], v[ro[3]]});
      }
      std::stable_sort(rc.begin(), rc.end(), [](const std::array<int, 4>& a, const std::array<int, 4>& b) {
        return a[2] != b[2] ? a[2] < b[2] : a[3] < b[3];
      });
      SandOrient so{};
      so.nx = h.dA[ro[0]]; so.nxw = h.dW[ro[0]];
      so.ny = h.dA[ro[1]]; so.nyw = h.dW[ro[1]];
      so.nv = h.dA[ro[2]]; so.nvw = h.dW[ro[2]];
      so.nz = h.dA[ro[3]]; so.nzw = h.dW[ro[3]];
      so.p = p;
      so.nch = nch;
      std::vector<int> flat, off((size_t)so.nvw * so.nzw + 1, 0);
      for (auto& a : rc) {
        flat.insert(flat.end(), a.begin(), a.end());
        off[(size_t)a[2] * so.nzw + a[3] + 1]++;
      }
      int npair = 0;
      for (size_t i = 1; i < off.size(); ++i) { npair += off[i] > 0; off[i] += off[i - 1]; }
      if (o == FWD) sd.n_ld = npair;
      int* d_ch = (int*)env->al.get(std::max<size_t>(flat.size(), 4) * sizeof(int));
      int* d_off = (int*)env->al.get(off.size() * sizeof(int));
      sd.bufs.push_back(d_ch);
      sd.bufs.push_back(d_off);
      if (!flat.empty()) FP_CUDA(cudaMemcpyAsync(d_ch, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice, env->stream));
      FP_CUDA(cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, env->stream));
      size_t per = (size_t)so.nx * so.ny * so.nv * so.nz * p;
      void* d_ar = env->al.get(per * env->elem);
      void* d_aw = env->al.get(std::max<size_t>(per * nch, 1) * env->elem);
      sd.bufs.push_back(d_ar);
      sd.bufs.push_back(d_aw);
      const char* A = (const char*)env->peps + h.offA * env->elem;
      const char* W = (const char*)env->pepo[layer] + h.offW * env->elem;
      if (env->elem == 8)
        sandwich_prepare<double>(env->stream, (const double*)A, h.dA, (const double*)W, h.dW, ro, d_ch, nch,
                                 (double*)d_aw, (double*)d_ar);
      else
        sandwich_prepare<float>(env->stream, (const float*)A, h.dA, (const float*)W, h.dW, ro, d_ch, nch,
                                (float*)d_aw, (float*)d_ar);
      so.d_ch = d_ch;
      so.d_pair_off = d_off;
      so.d_aw = d_aw;
      so.d_ar = d_ar;
      if (env->elem == 4 && sandwich_tc_fits(so)) {   // operand images of the tcgen05 sandwich
        size_t nk = 0, nb = 0;
        sandwich_tc_image_floats(so, &nk, &nb);
        void* ki = env->al.get(nk * sizeof(float));
        void* bi = env->al.get(nb * sizeof(float));
        sd.bufs.push_back(ki);
        sd.bufs.push_back(bi);
        sandwich_tc_images(env->stream, so, (float*)ki, (float*)bi);
        so.d_kimg = ki;
        so.d_arimg = bi;
      }
      sd.o[o] = so;
      // keep the host copy alive until the copies above have executed
      FP_CUDA(cudaStreamSynchronize(env->stream));
    }
  }
}

// ------------------------------------------------------------------ engine
template <class T>
struct Engine : EngineBase {
  fpeps_env* env;
  cudaStream_t s;
  int mode;   // fpeps_precision
  double flops = 0.0;
  double trunc_num = 0.0, trunc_den = 0.0;
  size_t budget_elems = (size_t)1 << 30;   // per-chunk intermediate size (elements)
  // true while an application runs entirely on the CUDA cores (FP32, round to
  // nearest): the reference columns of a scale calibration (see apply())
  bool simt_only = false;
  void* scr[2] = {nullptr, nullptr};
  size_t scr_n[2] = {0, 0};
  void* tc_scr = nullptr;
  size_t tc_n = 0;
  bool tc_used = false;

  // optional per-phase wall times (FPEPS_TRACE=1): synchronises around each phase
  bool trace = false;
  double ph[6] = {0, 0, 0, 0, 0, 0};   // apply, qr, svd, sketch, small, total
  struct Phase {
    Engine* e;
    int i;
    std::chrono::steady_clock::time_point t0;
    Phase(Engine* en, int idx) : e(en), i(idx) {
      if (e->trace) {
        cudaStreamSynchronize(e->s);
        t0 = std::chrono::steady_clock::now();
      }
    }
    ~Phase() {
      if (e->trace) {
        cudaStreamSynchronize(e->s);
        e->ph[i] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      }
    }
  };

  explicit Engine(fpeps_env* e) : env(e), s(e->stream), mode(e->cfg.prec) {
    if (const char* b = getenv("FPEPS_CHUNK_ELEMS")) budget_elems = (size_t)atoll(b);
    if (const char* t = getenv("FPEPS_TRACE")) trace = atoi(t) != 0;
  }
  ~Engine() override {
    for (int i = 0; i < 2; ++i)
      if (scr[i]) env->al.put(scr[i]);
    if (tc_scr) env->al.put(tc_scr);
  }

  T* scratch(int i, size_t n) {
    if (scr_n[i] < n) {
      if (scr[i]) env->al.put(scr[i]);
      scr[i] = env->al.get(n * sizeof(T));
      scr_n[i] = n;
    }
    return (T*)scr[i];
  }

  // ---------------------------------------------------------------- GEMMs
  // C = A B^T, A [M][lda], B [N][ldb], both k-contiguous
  // count = false for the products of the QR / SVD steps, which the algorithmic
  // flop count of the contraction leaves out
  void big_gemm(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B, int64_t ldb, T* C, OutMap om,
                bool count = true) {
    if (count) flops += 2.0 * (double)M * (double)N * (double)K;
    // tensor cores for every contraction with at least one full 128x128x32 tile and
    // 16-byte aligned rows; smaller edge contractions stay on the CUDA cores (FP32)
    if (sizeof(T) == 4 && (mode == FPEPS_TF32X3 || mode == FPEPS_BF16X3) && !simt_only &&
        gemm_tc_supported(M, N, K, lda, ldb) &&
        ((uintptr_t)A % 16) == 0 && ((uintptr_t)B % 16) == 0) {
      size_t need = gemm_tc_scratch_bytes(mode, M, N, K);
      if (!tc_scr || tc_n < need) {
        if (tc_scr) {
          check_tc();   // keep a recorded timeout before the error word is replaced
          env->al.put(tc_scr);
        }
        tc_scr = env->al.get(std::max<size_t>(need, 256));
        tc_n = std::max<size_t>(need, 256);
        FP_CUDA(cudaMemsetAsync(tc_scr, 0, sizeof(int), s));
      }
      gemm_tc(s, mode, M, N, K, (const float*)A, lda, (const float*)B, ldb, (float*)C, om, tc_scr, tc_n);
      tc_used = true;
      return;
    }
    gemm_simt<T>(s, M, N, K, T(1), A, lda, 1, B, ldb, 1, T(0), C, om);
  }

  // column-major C (m x n, ldc) = op(A) op(B), alpha/beta (small products, CUDA cores)
  void mm(int64_t m, int64_t n, int64_t k, T alpha, const T* A, bool ta, int64_t lda, const T* B, bool tb,
          int64_t ldb, T beta, T* C, int64_t ldc) {
    int64_t am = ta ? lda : 1, ak = ta ? 1 : lda;
    int64_t bn = tb ? 1 : ldb, bk = tb ? ldb : 1;
    gemm_simt<T>(s, m, n, k, alpha, A, am, ak, B, bn, bk, beta, C, out_colmajor(m, n, ldc));
  }
  // out (m x n, col-major, ld ldo) = X (m x k, col-major, ld ldx) S (k x n, col-major, ld lds): a tall
  // matrix times a small one. In 3xTF32 mode with at least one full tile this runs on the tensor
  // cores through K-major copies (X transposed, S with its rows padded to a multiple of 4).
  // The truncating FP32 accumulation of the tensor cores scales every column of the result by
  // 1 - beta_j, with beta_j set by the number of nonzero terms it sums (see apply()). Products
  // whose scale reaches the contracted value are therefore made unbiased:
  //   TALL_CALIBRATED  (S dense, so beta_j is the same for every column) the first two columns
  //                    are recomputed on the CUDA cores and the result divided by the fitted factor;
  //   TALL_CUDA_CORES  the whole product on the CUDA cores (FP32, round to nearest).
  enum Tall { TALL_PLAIN = 0, TALL_CALIBRATED = 1, TALL_CUDA_CORES = 2 };
  void mm_right(int64_t m, int n, int k, const T* X, int64_t ldx, const T* S, int64_t lds, T* out, int64_t ldo,
                int how = TALL_PLAIN) {
    const int kp = (k + 3) & ~3;
    if (how == TALL_CALIBRATED && n <= kCalCols) how = TALL_CUDA_CORES;
    if (sizeof(T) == 4 && (mode == FPEPS_TF32X3 || mode == FPEPS_BF16X3) && how != TALL_CUDA_CORES && !simt_only &&
        gemm_tc_supported(m, n, k, kp, kp)) {
      Arena ar = arena();
      T* Xt = ar.get_n<T>((size_t)m * kp);
      transpose_pad<T>(s, X, k, m, ldx, Xt, kp);
      T* St = ar.get_n<T>((size_t)n * kp);
      if (kp != k) FP_CUDA(cudaMemsetAsync(St, 0, sizeof(T) * n * kp, s));
      FP_CUDA(cudaMemcpy2DAsync(St, sizeof(T) * kp, S, sizeof(T) * lds, sizeof(T) * k, n, cudaMemcpyDeviceToDevice, s));
      big_gemm(m, n, k, Xt, kp, St, kp, out, out_colmajor(m, n, ldo), false);
      if (how == TALL_CALIBRATED) {
        T* ref = ar.get_n<T>((size_t)m * kCalCols);
        mm(m, kCalCols, k, T(1), X, false, ldx, S, false, lds, T(0), ref, m);
        double* alpha = env->d_scal + 6;
        if (ldo == m) {
          scale_against<T>(s, out, ref, m * kCalCols, alpha);
          scale_by_inv<T>(s, out, m * n, alpha);
        } else {   // strided output: fit on the first column, rescale column by column
          scale_against<T>(s, out, ref, m, alpha);
          for (int j = 0; j < n; ++j) scale_by_inv<T>(s, out + (int64_t)j * ldo, m, alpha);
        }
      }
      return;
    }
    mm(m, n, k, T(1), X, false, ldx, S, false, lds, T(0), out, ldo);
  }
  // Orthogonal projector onto the complement of the columns of Vm (n x a, col-major,
  // orthonormal columns). In 3xTF32 mode both products run on the tensor cores:
  // P = Vm^T X as a K-major product (Vm's columns and X's columns are contiguous),
  // then Vm P through a K-major copy VmT [n][ap] made once per projector.
  struct Projector {
    const T* Vm = nullptr;
    T* VmT = nullptr;
    int64_t n = 0;
    int a = 0, ap = 0;
    bool tc = false;
  };
  Projector projector(Arena& ar, const T* Vm, int64_t n, int a) {
    Projector P;
    P.Vm = Vm;
    P.n = n;
    P.a = a;
    P.ap = (a + 3) & ~3;
    P.tc = sizeof(T) == 4 && (mode == FPEPS_TF32X3 || mode == FPEPS_BF16X3) && a >= 1 && gemm_tc_supported(a, 1, n, n, n) &&
           gemm_tc_supported(n, 1, P.ap, P.ap, P.ap) && ((uintptr_t)Vm % 16) == 0;
    if (P.tc) {
      P.VmT = ar.get_n<T>((size_t)n * P.ap);
      transpose_pad<T>(s, Vm, a, n, n, P.VmT, P.ap);
    }
    return P;
  }
  // out (n x kk, col-major) = X - Vm (Vm^T X); out may alias X; tmp holds a x kk
  void project_out(const Projector& P, const T* X, T* out, int64_t kk, T* tmp) {
    if (P.tc && ((uintptr_t)X % 16) == 0) {
      Arena ar = arena();
      T* Pm = ar.get_n<T>((size_t)P.ap * kk);
      if (P.ap != P.a) FP_CUDA(cudaMemsetAsync(Pm, 0, sizeof(T) * P.ap * kk, s));
      big_gemm(P.a, kk, P.n, P.Vm, P.n, X, P.n, Pm, out_colmajor(P.a, kk, P.ap), false);
      T* R = ar.get_n<T>((size_t)P.n * kk);
      big_gemm(P.n, kk, P.ap, P.VmT, P.ap, Pm, P.ap, R, out_colmajor(P.n, kk, P.n), false);
      sub_into<T>(s, out, X, R, P.n * kk);
      return;
    }
    mm(P.a, kk, P.n, T(1), P.Vm, true, P.n, X, false, P.n, T(0), tmp, P.a);
    if (out != X) FP_CUDA(cudaMemcpyAsync(out, X, sizeof(T) * P.n * kk, cudaMemcpyDeviceToDevice, s));
    mm(P.n, kk, P.a, T(-1), P.Vm, false, P.n, tmp, false, P.a, T(1), out, P.n);
  }
  void mm64(int64_t m, int64_t n, int64_t k, const double* A, bool ta, int64_t lda, const double* B, bool tb,
            int64_t ldb, double* C, int64_t ldc) {
    int64_t am = ta ? lda : 1, ak = ta ? 1 : lda;
    int64_t bn = tb ? 1 : ldb, bk = tb ? ldb : 1;
    gemm_simt<double>(s, m, n, k, 1.0, A, am, ak, B, bn, bk, 0.0, C, out_colmajor(m, n, ldc));
  }

  // ---------------------------------------------------------------- site operators
  struct Site {
    int c = 0, t = 1, tp = 1;
    int bL = 1, bU = 1, bR = 1, bD = 1;
    int nA[4] = {1, 1, 1, 1}, nW[4] = {1, 1, 1, 1};   // ket and PEPO dims of the legs l, u, r, d
    const T *Tm = nullptr, *Tt = nullptr, *Tp = nullptr, *Tq = nullptr;
    const SiteSand* sd = nullptr;
  };
  struct Env3 {   // environment: [a][bond][bundle] and [bond][bundle][a]
    int a = 1;
    const T* E = nullptr;
    const T* Et = nullptr;
  };

  // error word of the tensor-core kernels (first int of tc_scr)
  int* tc_err() {
    if (!tc_scr) {
      tc_scr = env->al.get(256);
      tc_n = 256;
      FP_CUDA(cudaMemsetAsync(tc_scr, 0, sizeof(int), s));
    }
    tc_used = true;
    return (int*)tc_scr;
  }

  // the sandwich step: tcgen05 tensor cores (3xTF32) in the split-precision modes
  // when the site fits the tile, CUDA cores otherwise
  void sandwich(const SandOrient& o, int64_t nt, int64_t nk, const T* in, int64_t i_t, int64_t i_k, int64_t i_X,
                int64_t i_Y, T* out, int64_t o_t, int64_t o_k, int64_t o_V, int64_t o_Z) {
    const bool split = sizeof(T) == 4 && (mode == FPEPS_TF32X3 || mode == FPEPS_BF16X3) && !simt_only;
    if (split && o.d_kimg && sandwich_tc_fits(o)) {
      sandwich_apply_tcgen05(s, o, nt, nk, (const float*)in, i_t, i_k, i_X, i_Y, (float*)out, o_t, o_k, o_V, o_Z,
                             tc_err());
      return;
    }
    if (split && sandwich_mma_fits(o)) {
      sandwich_apply_tc(s, o, nt, nk, (const float*)in, i_t, i_k, i_X, i_Y, (float*)out, o_t, o_k, o_V, o_Z);
      return;
    }
    sandwich_apply<T>(s, o, nt, nk, in, i_t, i_k, i_X, i_Y, out, o_t, o_k, o_V, o_Z);
  }

  double sand_flops(const SandOrient& o, int64_t blocks, int n_ld) const {
    double ket = 2.0 * o.nch * (double)o.nx * o.nx * o.ny * o.ny * o.nv * o.nz * o.p;
    double bra = 2.0 * n_ld * (double)o.nv * o.nv * o.nz * o.nz * o.nx * o.ny * o.p;
    return (ket + bra) * (double)blocks;
  }
  int n_pairs(const SandOrient& o) {
    std::vector<int> off((size_t)o.nvw * o.nzw + 1);
    FP_CUDA(cudaMemcpy(off.data(), o.d_pair_off, off.size() * sizeof(int), cudaMemcpyDeviceToHost));
    int n = 0;
    for (size_t i = 1; i < off.size(); ++i) n += off[i] > off[i - 1];
    return n;
  }

  int64_t chunk_k(int64_t k, int64_t per_k) const {
    int64_t kc = (int64_t)(budget_elems / (size_t)std::max<int64_t>(per_k, 1));
    return std::max<int64_t>(1, std::min<int64_t>(k, kc));
  }

  // Y[k][Dn][a] = Theta_c X,  X[k][R][t']
  void theta(const Site& st, const Env3& el, const T* X, T* Y, int64_t k) {
    Phase ph_(this, 0);
    const int64_t t = st.t, tp = st.tp, U = st.bU, R = st.bR, L = st.bL, Dn = st.bD, a = el.a;
    const SandOrient& o = st.sd->o[FWD];
    const int64_t kc = chunk_k(k, t * std::max(U * R, L * Dn));
    T* G1 = scratch(0, (size_t)(t * kc * U * R));
    T* G2 = scratch(1, (size_t)(t * kc * L * Dn));
    for (int64_t k0 = 0; k0 < k; k0 += kc) {
      const int64_t kk = std::min(kc, k - k0);
      big_gemm(t * U, kk * R, tp, st.Tm, tp, X + k0 * R * tp, tp, G1, OutMap{U, kk * U * R, R, R, U * R, 1});
      {
        const double sf = sand_flops(o, t * kk, st.sd->n_ld);
        ProfToken pt = prof_begin(PROF_SANDWICH, s, sf, (double)sizeof(T) * t * kk * (double)(U * R + L * Dn));
        sandwich(o, t, kk, G1, kk * U * R, U * R, R, 1, G2, L, Dn * t * L, 1, t * L);
        prof_end(pt, s);
        flops += sf;
      }
      big_gemm(a, kk * Dn, t * L, el.E, t * L, G2, t * L, Y + k0 * Dn * a, OutMap{a, 0, 1, Dn, Dn * a, a});
    }
  }
  // Z[k][R][t'] = Theta_c^T Y,  Y[k][Dn][a]
  void theta_t(const Site& st, const Env3& el, const T* Y, T* Z, int64_t k) {
    Phase ph_(this, 0);
    const int64_t t = st.t, tp = st.tp, U = st.bU, R = st.bR, L = st.bL, Dn = st.bD, a = el.a;
    const SandOrient& o = st.sd->o[BWD];
    const int64_t kc = chunk_k(k, t * std::max(U * R, L * Dn));
    T* H1 = scratch(0, (size_t)(t * kc * L * Dn));
    T* H2 = scratch(1, (size_t)(t * kc * U * R));
    for (int64_t k0 = 0; k0 < k; k0 += kc) {
      const int64_t kk = std::min(kc, k - k0);
      big_gemm(t * L, kk * Dn, a, el.Et, a, Y + k0 * Dn * a, a, H1, OutMap{L, kk * L * Dn, Dn, Dn, L * Dn, 1});
      {
        const double sf = sand_flops(o, t * kk, st.sd->n_ld);
        ProfToken pt = prof_begin(PROF_SANDWICH, s, sf, (double)sizeof(T) * t * kk * (double)(U * R + L * Dn));
        sandwich(o, t, kk, H1, kk * L * Dn, L * Dn, Dn, 1, H2, U, R * t * U, 1, t * U);
        prof_end(pt, s);
        flops += sf;
      }
      big_gemm(tp, kk * R, t * U, st.Tt, t * U, H2, t * U, Z + k0 * R * tp, OutMap{tp, 0, 1, R, R * tp, tp});
    }
  }
  // Z[k][L][t] = ThetaR_c X,  X[k][Dn][a_c]; er = environment to the right of site c
  void theta_r(const Site& st, const Env3& er, const T* X, T* Z, int64_t k) {
    Phase ph_(this, 0);
    const int64_t t = st.t, tp = st.tp, U = st.bU, R = st.bR, L = st.bL, Dn = st.bD, a = er.a;
    const SandOrient& o = st.sd->o[RF];
    const int64_t kc = chunk_k(k, tp * std::max(R * Dn, L * U));
    T* W1 = scratch(0, (size_t)(tp * kc * R * Dn));
    T* W2 = scratch(1, (size_t)(tp * kc * L * U));
    for (int64_t k0 = 0; k0 < k; k0 += kc) {
      const int64_t kk = std::min(kc, k - k0);
      big_gemm(tp * R, kk * Dn, a, er.Et, a, X + k0 * Dn * a, a, W1, OutMap{R, kk * R * Dn, Dn, Dn, R * Dn, 1});
      {
        const double sf = sand_flops(o, tp * kk, st.sd->n_ld);
        ProfToken pt = prof_begin(PROF_SANDWICH, s, sf, (double)sizeof(T) * tp * kk * (double)(U * R + L * Dn));
        sandwich(o, tp, kk, W1, kk * R * Dn, R * Dn, Dn, 1, W2, U, L * tp * U, tp * U, 1);
        prof_end(pt, s);
        flops += sf;
      }
      big_gemm(t, kk * L, tp * U, st.Tp, tp * U, W2, tp * U, Z + k0 * L * t, OutMap{t, 0, 1, L, L * t, t});
    }
  }
  // X[k][Dn][a_c] = ThetaR_c^T Z,  Z[k][L][t]
  void theta_r_t(const Site& st, const Env3& er, const T* Z, T* X, int64_t k) {
    Phase ph_(this, 0);
    const int64_t t = st.t, tp = st.tp, U = st.bU, R = st.bR, L = st.bL, Dn = st.bD, a = er.a;
    const SandOrient& o = st.sd->o[RB];
    const int64_t kc = chunk_k(k, tp * std::max(R * Dn, L * U));
    T* W1 = scratch(0, (size_t)(tp * kc * L * U));
    T* W2 = scratch(1, (size_t)(tp * kc * R * Dn));
    for (int64_t k0 = 0; k0 < k; k0 += kc) {
      const int64_t kk = std::min(kc, k - k0);
      big_gemm(tp * U, kk * L, t, st.Tq, t, Z + k0 * L * t, t, W1, OutMap{U, kk * L * U, 1, L, L * U, U});
      {
        const double sf = sand_flops(o, tp * kk, st.sd->n_ld);
        ProfToken pt = prof_begin(PROF_SANDWICH, s, sf, (double)sizeof(T) * tp * kk * (double)(U * R + L * Dn));
        sandwich(o, tp, kk, W1, kk * L * U, L * U, U, 1, W2, R, Dn * tp * R, 1, tp * R);
        prof_end(pt, s);
        flops += sf;
      }
      big_gemm(a, kk * Dn, tp * R, er.E, tp * R, W2, tp * R, X + k0 * Dn * a, OutMap{a, 0, 1, Dn, Dn * a, a});
    }
  }

  // ---------------------------------------------------------------- calibrated applications
  // The tensor cores add every MMA's products into the FP32 accumulator with
  // truncation toward zero. Errors of that kind do not average out: each one
  // shrinks the partial sum it rounds, so a tensor-core application returns the
  // exact result times a common factor 1 - beta (measured on GB300: beta ~ 1.5e-6
  // per 256-term accumulation chunk of the GEMM, 2e-6 to 6e-6 for a whole Theta_c
  // application), and the contracted value, a product of one application per site
  // and row, inherits the sum of those betas. Subspace iterations and the CBE
  // expansion are insensitive to a common factor; the applications whose scale
  // reaches the value (the fitted environments and tensors, the last zip-up
  // application of a pass without fit, the closing row) are calibrated: the same
  // application runs for the first kCalCols vectors on the CUDA cores (FP32 with
  // round-to-nearest, unbiased), the least-squares factor
  // alpha = <y_tc, y_ref> / <y_ref, y_ref> over those columns is formed on the
  // device, and the whole output is divided by it. An application with at most
  // kCalCols vectors runs on the CUDA cores outright.
  static constexpr int kCalCols = 2;
  enum Op { OP_THETA = 0, OP_THETA_T = 1, OP_THETA_R = 2, OP_THETA_R_T = 3 };
  void run_op(int op, const Site& st, const Env3& e, const T* in, T* out, int64_t k) {
    switch (op) {
      case OP_THETA: theta(st, e, in, out, k); break;
      case OP_THETA_T: theta_t(st, e, in, out, k); break;
      case OP_THETA_R: theta_r(st, e, in, out, k); break;
      default: theta_r_t(st, e, in, out, k); break;
    }
  }
  int64_t op_out_size(int op, const Site& st, const Env3& e) const {
    switch (op) {
      case OP_THETA: return (int64_t)st.bD * e.a;
      case OP_THETA_T: return (int64_t)st.bR * st.tp;
      case OP_THETA_R: return (int64_t)st.bL * st.t;
      default: return (int64_t)st.bD * e.a;
    }
  }
  void apply(int op, const Site& st, const Env3& e, const T* in, T* out, int64_t k, bool calibrate) {
    const bool tc = sizeof(T) == 4 && (mode == FPEPS_TF32X3 || mode == FPEPS_BF16X3);
    if (!calibrate || !tc || simt_only) {
      run_op(op, st, e, in, out, k);
      return;
    }
    const double f0 = flops;
    if (k <= kCalCols) {
      simt_only = true;
      run_op(op, st, e, in, out, k);
      simt_only = false;
      return;
    }
    run_op(op, st, e, in, out, k);
    const int64_t nout = op_out_size(op, st, e);
    Arena ar = arena();
    T* ref = ar.get_n<T>((size_t)kCalCols * nout);
    const double f1 = flops;
    simt_only = true;
    run_op(op, st, e, in, ref, kCalCols);   // inputs are [k][...]: the first kCalCols vectors
    simt_only = false;
    flops = f1;                              // the reference is not algorithmic work
    double* alpha = env->d_scal + 4;
    scale_against<T>(s, out, ref, (int64_t)kCalCols * nout, alpha);
    scale_by_inv<T>(s, out, k * nout, alpha);
    (void)f0;
  }

  // ---------------------------------------------------------------- helpers
  Arena arena() { Arena ar; ar.al = &env->al; return ar; }

  double host_norm(const T* x, int64_t n) {
    frob_norm_f64<T>(s, x, n, env->d_scal);
    FP_CUDA(cudaMemcpyAsync(env->h_scal, env->d_scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    FP_CUDA(cudaStreamSynchronize(s));
    check_tc();
    double v = env->h_scal[0];
    FP_CHECK(std::isfinite(v), FPEPS_ERR_NUMERIC, "non-finite norm");
    return v;
  }
  // the tensor-core kernels record a bounded-wait timeout in their error word
  void check_tc() {
    if (!tc_used) return;
    FP_CUDA(cudaMemcpyAsync(env->h_info + 1, tc_scr, sizeof(int), cudaMemcpyDeviceToHost, s));
    FP_CUDA(cudaStreamSynchronize(s));
    if (env->h_info[1]) throw Error{FPEPS_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait timed out"};
  }
  int read_info() {
    FP_CUDA(cudaMemcpyAsync(env->h_info, env->d_info, sizeof(int), cudaMemcpyDeviceToHost, s));
    FP_CUDA(cudaStreamSynchronize(s));
    check_tc();
    return env->h_info[0];
  }

  Site make_site(Arena& ar, int row, int c, bool need_fwd, bool need_r) {
    Site st;
    st.c = c;
    const SiteHost& h = env->sites[env->layer][row * env->cfg.Ly + c];
    st.bL = bund(h, 0); st.bU = bund(h, 1); st.bR = bund(h, 2); st.bD = bund(h, 3);
    for (int l = 0; l < 4; ++l) {
      st.nA[l] = h.dA[l];
      st.nW[l] = h.dW[l];
    }
    st.t = env->tb[c];
    st.tp = env->tb[c + 1];
    FP_CHECK(env->tphys[c] == st.bU, FPEPS_ERR_ARG, "boundary bundle does not match the row's up legs");
    st.sd = &env->sand[env->layer][row * env->cfg.Ly + c];
    const T* Tm = (const T*)env->T[c];
    st.Tm = Tm;
    const int64_t t = st.t, U = st.bU, tp = st.tp;
    // Tt and Tp meet the sandwich output's unit-stride bundle (U) in the GEMM after the
    // sandwich: their U index is PEPO-outermost like that output (see bundle_index)
    T* tmp = (need_fwd || need_r) ? ar.get_n<T>(t * U * tp) : nullptr;
    if (need_fwd) {
      T* Tt = ar.get_n<T>(t * U * tp);
      permute3<T>(s, Tm, tmp, t, U, tp, 2, 0, 1);
      bundle_outer<T>(s, tmp, Tt, tp * t, h.dA[1], h.dW[1]);
      st.Tt = Tt;
    }
    if (need_r) {
      T* Tp = ar.get_n<T>(t * U * tp);
      T* Tq = ar.get_n<T>(t * U * tp);
      permute3<T>(s, Tm, tmp, t, U, tp, 0, 2, 1);
      bundle_outer<T>(s, tmp, Tp, t * tp, h.dA[1], h.dW[1]);
      permute3<T>(s, Tm, Tq, t, U, tp, 2, 1, 0);
      st.Tp = Tp;
      st.Tq = Tq;
    }
    return st;
  }

  // env tensors from a vector block V[a][bundle][bond] (a vectors): E [a][bond][bundle], Et
  // [bond][bundle][a]. E meets the sandwich output in the GEMM after the sandwich, so its bundle
  // (ket dim n, PEPO dim nw) is stored PEPO-outermost like that output (see bundle_index).
  Env3 env_from_vectors(Arena& ar, const T* Vb, int a, int64_t bundle, int64_t bond, int n, int nw) {
    Env3 e;
    e.a = a;
    T* E = ar.get_n<T>((int64_t)a * bundle * bond);
    T* Et = ar.get_n<T>((int64_t)a * bundle * bond);
    Arena tmp = arena();
    T* En = tmp.get_n<T>((int64_t)a * bundle * bond);
    permute3<T>(s, Vb, En, a, bundle, bond, 0, 2, 1);
    bundle_outer<T>(s, En, E, (int64_t)a * bond, n, nw);
    permute3<T>(s, Vb, Et, a, bundle, bond, 2, 1, 0);
    e.E = E;
    e.Et = Et;
    return e;
  }
  Env3 unit_env(Arena& ar) {
    T* one = ar.get_n<T>(1);
    fill<T>(s, one, 1, T(1));
    Env3 e;
    e.a = 1;
    e.E = one;
    e.Et = one;
    return e;
  }

  // ---------------------------------------------------------------- QR (Sec. IV)
  // Y (m x k, col-major, ld = m, m >= k) = Q R. CholeskyQR2 in FP64 (Gram,
  // Cholesky, Q = Y R^-1, twice). Columns are orthonormalised in their order; a
  // column whose Cholesky pivot (squared residual against the columns before it)
  // is at most 1e-13 of the largest squared column norm depends numerically on
  // them and gives a zero column of Q and a zero row of R. R: k x k row-major
  // FP64, or null.
  // How Q = Y R^-1 is formed in one pass: PASS_PLAIN on the tensor cores (3xTF32 mode);
  // PASS_CUDA_CORES unbiased on the CUDA cores; PASS_DIAG_SPLIT the diagonal of R^-1 as an
  // FP32 column scaling (round to nearest) plus the off-diagonal rest on the tensor cores. In
  // the second pass R is the identity up to the first pass's rounding, so the rest is small
  // and so is the truncation error of its accumulation: the columns of Q keep unit norm.
  enum Pass { PASS_PLAIN = 0, PASS_CUDA_CORES = 1, PASS_DIAG_SPLIT = 2 };
  void one_pass(Arena& ar, const T* Y, int64_t m, int k, T* Q, double* R, int how = PASS_PLAIN) {
    double* G = ar.get_n<double>((int64_t)k * k);
    gram_f64<T>(s, Y, m, k, m, G);
    cholesky_upper_f64(s, G, k, env->d_info, ar.get_n<double>(8));
    FP_CHECK(read_info() == 0, FPEPS_ERR_NUMERIC, "QR: non-finite Gram matrix");
    T* Bt = ar.get_n<T>((int64_t)k * k);
    double* Rinv = ar.get_n<double>((int64_t)k * k);
    tri_inverse_upper_f64(s, G, k, Rinv);
    convert_f64_t<T>(s, Rinv, k, k, Bt);   // Rinv is row-major; Bt col-major
    // Q(m, j) = sum_i Y(m, i) Rinv(i, j)
    if (how == PASS_DIAG_SPLIT) {
      zero_diag<T>(s, Bt, k, k);
      mm_right(m, k, k, Y, m, Bt, k, Q, m);
      add_diag_cols<T>(s, Y, m, k, m, Rinv, k, Q, m);
    } else {
      mm_right(m, k, k, Y, m, Bt, k, Q, m, how == PASS_CUDA_CORES ? TALL_CUDA_CORES : TALL_PLAIN);
    }
    if (R) FP_CUDA(cudaMemcpyAsync(R, G, sizeof(double) * k * k, cudaMemcpyDeviceToDevice, s));
  }

  // Thin QR (CholeskyQR2). The first pass's rounding is absorbed by the second when only Q
  // is needed; when R is returned too (the singular values come from it) the first pass is
  // unbiased as well, so that Q R reproduces Y.
  void qr(const T* Y, int64_t m, int k, T* Q, double* R) {
    Phase ph_(this, 1);
    Arena ar = arena();
    T* Q1 = ar.get_n<T>(m * k);
    double* R1 = R ? ar.get_n<double>((int64_t)k * k) : nullptr;
    double* R2 = R ? ar.get_n<double>((int64_t)k * k) : nullptr;
    one_pass(ar, Y, m, k, Q1, R1, R ? PASS_CUDA_CORES : PASS_PLAIN);
    one_pass(ar, Q1, m, k, Q, R2, PASS_DIAG_SPLIT);
    if (R) {   // R = R2 R1 (row-major)
      gemm_simt<double>(s, k, k, k, 1.0, R2, k, 1, R1, 1, k, 0.0, R, out_rowmajor(k, k, k));
    }
  }

  // A basis of col(Y) for the next step of the subspace iteration: one CholeskyQR pass,
  // Y R1^-1. Its columns are orthonormal only to O(cond(Y)^2 u), but it equals the two-pass Q
  // times an upper-triangular matrix with a positive diagonal (R2), and Gram-Schmidt in
  // column order is invariant under such a factor: every later orthonormalisation, and so
  // the final Q, is the same as with two passes here, up to rounding.
  void qr_basis(const T* Y, int64_t m, int k, T* Q) {
    Phase ph_(this, 1);
    Arena ar = arena();
    one_pass(ar, Y, m, k, Q, nullptr, PASS_PLAIN);
  }

  // ---------------------------------------------------------------- rSVD (Sec. IV)
  struct Lin {
    int64_t m, n;
    std::function<void(const T*, T*, int64_t)> fwd, bwd;
    // the last application B^T = A^T Q, whose scale reaches the singular values
    // (empty: bwd)
    std::function<void(const T*, T*, int64_t)> bwd_last;
  };
  struct RsvdOut {
    T* Q;        // m x k
    T* QbW;      // n x k  right singular vectors (sorted)
    double* U;   // k x k  left singular vectors in the Q basis, col-major (sorted)
    std::vector<double> sigma;
  };
  // Randomized subspace iteration with re-orthonormalisation after every
  // application (one CholeskyQR pass for the intermediate bases, two for the last),
  // then B = Q^T A = R_b^T Q_b^T and the Jacobi SVD of R_b^T.
  RsvdOut rsvd(Arena& ar, Lin& A, const T* omega, int k, int q) {
    RsvdOut r;
    const int64_t m = A.m, n = A.n;
    T* Y = ar.get_n<T>(m * k);
    T* Z = ar.get_n<T>(n * k);
    r.Q = ar.get_n<T>(m * k);
    T* Qz = ar.get_n<T>(n * k);
    // intermediate bases of the iteration take one CholeskyQR pass (qr_basis), the last Q two
    A.fwd(omega, Y, k);
    if (q > 0) qr_basis(Y, m, k, r.Q);
    else qr(Y, m, k, r.Q, nullptr);
    for (int it = 0; it < q; ++it) {
      A.bwd(r.Q, Z, k);
      qr_basis(Z, n, k, Qz);
      A.fwd(Qz, Y, k);
      if (it + 1 < q) qr_basis(Y, m, k, r.Q);
      else qr(Y, m, k, r.Q, nullptr);
    }
    (A.bwd_last ? A.bwd_last : A.bwd)(r.Q, Z, k);   // B^T = A^T Q  (n x k)
    double* Rb = ar.get_n<double>((int64_t)k * k);
    qr(Z, n, k, Qz, Rb);                    // B^T = Q_b R_b
    // SVD of R_b^T: the row-major R_b array read as col-major is R_b^T
    double* Ms = ar.get_n<double>((int64_t)k * k);
    FP_CUDA(cudaMemcpyAsync(Ms, Rb, sizeof(double) * k * k, cudaMemcpyDeviceToDevice, s));
    double* Uj = ar.get_n<double>((int64_t)k * k);
    double* Vj = ar.get_n<double>((int64_t)k * k);
    double* sg = ar.get_n<double>(k);
    int* order = ar.get_n<int>(k);
    {
      Phase ph_(this, 2);
      svd_jacobi_f64(s, Ms, k, Uj, sg, Vj, order, env->d_info, ar.get(64));
    }
    FP_CHECK(read_info() == 0, FPEPS_ERR_NUMERIC, "Jacobi SVD did not converge");
    r.U = Uj;
    double* Vs = ar.get_n<double>((int64_t)k * k);
    gather_cols_f64(s, Vj, order, k, Vs);
    T* Vt = ar.get_n<T>((int64_t)k * k);
    convert_f64<T>(s, Vs, Vt, (int64_t)k * k);
    r.QbW = ar.get_n<T>(n * k);
    mm_right(n, k, k, Qz, n, Vt, k, r.QbW, n, TALL_CALIBRATED);
    r.sigma.resize(k);
    FP_CUDA(cudaMemcpyAsync(r.sigma.data(), sg, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    FP_CUDA(cudaStreamSynchronize(s));
    return r;
  }

  // ---------------------------------------------------------------- row 0 / last row
  void first_row(fpeps_env* e, int row) override {
    const int Ly = e->cfg.Ly;
    std::vector<int> tb(Ly + 1, 1), ph(Ly, 1);
    std::vector<void*> T_new(Ly, nullptr);
    double log_s = 0.0;
    for (int c = 0; c < Ly; ++c) {
      const SiteHost& h = e->sites[e->layer][row * Ly + c];
      const int64_t nL = bund(h, 0), nD = bund(h, 3), nR = bund(h, 2);
      T* out = (T*)e->al.get(sizeof(T) * nL * nD * nR);
      const T* A = (const T*)((const char*)e->peps + h.offA * e->elem);
      const T* W = (const T*)((const char*)e->pepo[e->layer] + h.offW * e->elem);
      first_row_tensor<T>(s, A, h.dA, W, h.dW, out);
      double nrm = host_norm(out, nL * nD * nR);
      FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "row-0 site tensor is zero");
      scale_by_inv<T>(s, out, nL * nD * nR, e->d_scal);
      log_s += std::log(nrm);
      T_new[c] = out;
      tb[c] = (int)nL;
      tb[c + 1] = (int)nR;
      ph[c] = (int)nD;
    }
    for (void* p : e->T) e->al.put(p);
    e->T = T_new;
    e->tb = tb;
    e->tphys = ph;
    e->log_scale += log_s;
    if (e->cfg.symmetry == 1) {   // bond t_c of the exact row-0 boundary is the R bundle of site c
      e->qT.assign(Ly + 1, std::vector<int32_t>{0, 0});
      for (int c = 0; c < Ly - 1; ++c) e->qT[c + 1] = e->sites[e->layer][row * Ly + c].qB[2];
    }
  }

  void close_row(fpeps_env* e, int row) override {
    const int Ly = e->cfg.Ly;
    ensure_sandwich(e, e->layer, row);
    Arena keep = arena();
    Env3 v = unit_env(keep);
    T* ones = keep.get_n<T>(1);
    fill<T>(s, ones, 1, T(1));
    double log_s = 0.0, val = 0.0;
    for (int c = 0; c < Ly; ++c) {
      Arena ar = arena();
      Site st = make_site(ar, row, c, true, false);
      FP_CHECK(st.bD == 1, FPEPS_ERR_ARG, "last row must have dimension-1 down legs");
      T* Z = ar.get_n<T>((int64_t)st.bR * st.tp);
      apply(OP_THETA_T, st, v, ones, Z, 1, true);
      const int64_t n = (int64_t)st.bR * st.tp;
      if (c < Ly - 1) {
        double nrm = host_norm(Z, n);
        FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "closing vector vanished");
        scale_by_inv<T>(s, Z, n, e->d_scal);
        log_s += std::log(nrm);
        Arena nk = arena();
        Env3 nv = env_from_vectors(nk, Z, 1, st.bR, st.tp, st.nA[2], st.nW[2]);
        FP_CUDA(cudaStreamSynchronize(s));
        keep.reset();
        keep.live = nk.live;   // transfer ownership
        nk.live.clear();
        v = nv;
        T* o2 = keep.get_n<T>(1);
        fill<T>(s, o2, 1, T(1));
        ones = o2;
      } else {
        T hv;
        FP_CUDA(cudaMemcpyAsync(&hv, Z, sizeof(T), cudaMemcpyDeviceToHost, s));
        FP_CUDA(cudaStreamSynchronize(s));
        val = (double)hv;
      }
      FP_CUDA(cudaStreamSynchronize(s));
    }
    FP_CHECK(std::isfinite(val), FPEPS_ERR_NUMERIC, "non-finite closing value");
    e->value_sign = val >= 0 ? 1 : -1;
    e->value_log = e->log_scale + log_s + (val != 0 ? std::log(std::fabs(val)) : -INFINITY);
    e->have_value = true;
  }

  // ---------------------------------------------------------------- compression
  void compress(fpeps_env* e, int row, const fpeps_rsvd_params& prm, fpeps_stats* out) override {
    const int Ly = e->cfg.Ly;
    const int chi = e->cfg.chi;
    ensure_sandwich(e, e->layer, row);
    flops = 0.0;
    trunc_num = trunc_den = 0.0;
    for (double& v : ph) v = 0.0;
    const auto t_start = std::chrono::steady_clock::now();
    cudaEvent_t ev0, ev1;
    FP_CUDA(cudaEventCreate(&ev0));
    FP_CUDA(cudaEventCreate(&ev1));
    FP_CUDA(cudaEventRecord(ev0, s));
    e->spectra.zip.assign(Ly, {});
    e->spectra.fit.assign(Ly, {});

    const bool sym = e->cfg.symmetry == 1;
    if (sym) {
      FP_CHECK((int)e->qT.size() == Ly + 1, FPEPS_ERR_STATE, "charge sectors: the boundary carries no charges");
    }
    std::vector<std::vector<int32_t>> qnew(Ly + 1, std::vector<int32_t>{0, 0});
    std::vector<int32_t> qa{0, 0};               // charges of the new bond a_{c-1}
    Arena rowmem = arena();                      // lives for the whole row
    std::vector<T*> Nvec(Ly, nullptr);           // zip-up isometries as vectors [chi][Dn][a]
    std::vector<int> abond(Ly + 1, 1);           // new bonds
    std::vector<Env3> EL(Ly);
    std::vector<T*> ELvec(Ly, nullptr);
    EL[0] = unit_env(rowmem);
    double log_s = 0.0;
    const uint64_t w3 = (uint64_t)row | ((uint64_t)env->cur << 16);   // row | environment << 16

    // ---------------- zip-up, left to right
    for (int c = 0; c < Ly - 1; ++c) {
      Arena ar = arena();
      Site st = make_site(ar, row, c, true, false);
      const int a = EL[c].a;
      const int64_t rows = (int64_t)a * st.bD, cols = (int64_t)st.tp * st.bR;
      if (sym) {
        // Theta_c is block diagonal in the charge of the cut bond: rows (Dn, a) carry
        // q_a - Q_Dn, columns (R, t') carry q_t' + Q_R. rSVD per sector (sketch = the
        // dense Omega's rows of the sector's columns), one global truncation to chi.
        const SiteHost& hs = e->sites[e->layer][row * Ly + c];
        const std::vector<int32_t>& QD = hs.qB[3];
        const std::vector<int32_t>& QR = hs.qB[2];
        const std::vector<int32_t>& qt = e->qT[c + 1];
        FP_CHECK((int64_t)QD.size() == 2 * st.bD && (int64_t)QR.size() == 2 * st.bR &&
                     (int64_t)qt.size() == 2 * st.tp && (int64_t)qa.size() == 2 * a,
                 FPEPS_ERR_STATE, "charge sectors: charge lists do not match the bonds");
        std::vector<int32_t> rowq(2 * rows), colq(2 * cols);
        for (int64_t d = 0; d < st.bD; ++d)
          for (int64_t ai = 0; ai < a; ++ai)
            for (int t = 0; t < 2; ++t) rowq[2 * (d * a + ai) + t] = qa[2 * ai + t] - QD[2 * d + t];
        for (int64_t R = 0; R < st.bR; ++R)
          for (int64_t tq = 0; tq < st.tp; ++tq)
            for (int t = 0; t < 2; ++t) colq[2 * (R * st.tp + tq) + t] = qt[2 * tq + t] + QR[2 * R + t];
        std::vector<SecIdx> secs = sectors_of(ar, rowq, colq);
        const size_t ns = secs.size();
        std::vector<int> cap(ns), kq(ns);
        int kmax = 0;
        int64_t capsum = 0;
        for (size_t n = 0; n < ns; ++n) {
          const int64_t rank = std::min<int64_t>((int64_t)secs[n].ri.size(), (int64_t)secs[n].ci.size());
          cap[n] = (int)std::min<int64_t>(chi, rank);
          kq[n] = prm.exact_svd ? (int)rank : (int)std::min<int64_t>((int64_t)cap[n] + prm.oversample, rank);
          kmax = std::max(kmax, kq[n]);
          capsum += cap[n];
        }
        FP_CHECK(capsum > 0, FPEPS_ERR_NUMERIC, "charge sectors: rows and columns share no charge");
        T* omega = ar.get_n<T>(cols * kmax);
        int64_t perm[2] = {st.bR, st.tp};
        gaussian_sketch<T>(s, omega, cols, kmax, cols, perm, e->cfg.seed, (uint64_t)e->layer, (uint64_t)c, w3);
        T* fullc = ar.get_n<T>(cols * kmax);
        T* fullr = ar.get_n<T>(rows * kmax);
        Env3 elc = EL[c];
        double tot = 0.0;
        std::vector<T*> Ls(ns, nullptr), Rs(ns, nullptr);
        std::vector<std::vector<double>> sig(ns);
        std::vector<Pick> cand;
        for (size_t n = 0; n < ns; ++n) {
          const int64_t nr = (int64_t)secs[n].ri.size(), nc = (int64_t)secs[n].ci.size();
          const int64_t* dri = secs[n].d_ri;
          const int64_t* dci = secs[n].d_ci;
          T* om = ar.get_n<T>(nc * kq[n]);
          gather_rows<T>(s, omega, cols, dci, nc, kq[n], om, nc);
          Lin A{nr, nc,
                [&, dri, dci, nr, nc](const T* X, T* Y, int64_t kk) {
                  FP_CUDA(cudaMemsetAsync(fullc, 0, sizeof(T) * cols * kk, s));
                  scatter_rows<T>(s, X, nc, dci, nc, kk, fullc, cols);
                  theta(st, elc, fullc, fullr, kk);
                  gather_rows<T>(s, fullr, rows, dri, nr, kk, Y, nr);
                },
                [&, dri, dci, nr, nc](const T* Y, T* Z, int64_t kk) {
                  FP_CUDA(cudaMemsetAsync(fullr, 0, sizeof(T) * rows * kk, s));
                  scatter_rows<T>(s, Y, nr, dri, nr, kk, fullr, rows);
                  theta_t(st, elc, fullr, fullc, kk);
                  gather_rows<T>(s, fullc, cols, dci, nc, kk, Z, nc);
                },
                [&, dri, dci, nr, nc](const T* Y, T* Z, int64_t kk) {   // last application (see the dense zip-up)
                  FP_CUDA(cudaMemsetAsync(fullr, 0, sizeof(T) * rows * kk, s));
                  scatter_rows<T>(s, Y, nr, dri, nr, kk, fullr, rows);
                  apply(OP_THETA_T, st, elc, fullr, fullc, kk, prm.n_fit == 0);
                  gather_rows<T>(s, fullc, cols, dci, nc, kk, Z, nc);
                }};
          RsvdOut r = rsvd(ar, A, om, kq[n], prm.power_iters);
          T* Ut = ar.get_n<T>((int64_t)kq[n] * kq[n]);
          convert_f64<T>(s, r.U, Ut, (int64_t)kq[n] * kq[n]);
          Ls[n] = ar.get_n<T>(nr * kq[n]);
          mm_right(nr, kq[n], kq[n], r.Q, nr, Ut, kq[n], Ls[n], nr, TALL_CALIBRATED);
          Rs[n] = r.QbW;
          sig[n] = r.sigma;
          for (double v : r.sigma) tot += v * v;
          for (int j = 0; j < cap[n]; ++j) cand.push_back({-r.sigma[j], (int)n, j});
        }
        // global truncation: the chi_c largest over the sectors' offers (ties: sector
        // order, then index); kept triplets ordered by sector, then value
        const int chi_c = (int)std::min<int64_t>(chi, capsum);
        std::vector<Pick> kept = pick_global(cand, chi_c);
        T* N = rowmem.get_n<T>(rows * chi_c);
        T* elv = rowmem.get_n<T>(cols * chi_c);
        FP_CUDA(cudaMemsetAsync(N, 0, sizeof(T) * rows * chi_c, s));
        FP_CUDA(cudaMemsetAsync(elv, 0, sizeof(T) * cols * chi_c, s));
        std::vector<double> sv(chi_c), alive(chi_c);
        std::vector<int32_t> qk(2 * (size_t)chi_c);
        double kept2 = 0.0;
        for (int m = 0; m < chi_c; ++m) {
          const int n = kept[m].n, j = kept[m].j;
          const SecIdx& x = secs[n];
          const int64_t nr = (int64_t)x.ri.size(), nc = (int64_t)x.ci.size();
          scatter_rows<T>(s, Ls[n] + (int64_t)j * nr, nr, x.d_ri, nr, 1, N + (int64_t)m * rows, rows);
          scatter_rows<T>(s, Rs[n] + (int64_t)j * nc, nc, x.d_ci, nc, 1, elv + (int64_t)m * cols, cols);
          sv[m] = sig[n][j];
          kept2 += sv[m] * sv[m];
          alive[m] = (tot > 0 && sv[m] * sv[m] > 1e-30 * tot) ? 1.0 : 0.0;
          qk[2 * m] = x.q.first;
          qk[2 * m + 1] = x.q.second;
        }
        double* d_alive = ar.get_n<double>(chi_c);
        FP_CUDA(cudaMemcpyAsync(d_alive, alive.data(), sizeof(double) * chi_c, cudaMemcpyHostToDevice, s));
        scale_cols<T>(s, N, rows, chi_c, rows, d_alive);
        // sign gauge and remainder, as in the dense zip-up
        double* sgn = ar.get_n<double>(chi_c);
        T* gw = ar.get_n<T>(rows);
        int64_t gperm[2] = {st.bD, a};
        gaussian_sketch<T>(s, gw, rows, 1, rows, gperm, e->cfg.seed, (uint64_t)e->layer, (uint64_t)c | (2ull << 16),
                           w3);
        col_signs<T>(s, N, rows, chi_c, rows, gw, sgn);
        scale_cols<T>(s, N, rows, chi_c, rows, sgn);
        double* sc = ar.get_n<double>(chi_c);
        double* sgd = ar.get_n<double>(chi_c);
        FP_CUDA(cudaMemcpyAsync(sgd, sv.data(), sizeof(double) * chi_c, cudaMemcpyHostToDevice, s));
        mul_vec(s, sgd, sgn, sc, chi_c);
        scale_cols<T>(s, elv, cols, chi_c, cols, sc);
        double nrm = host_norm(elv, cols * chi_c);
        FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "zip-up remainder vanished");
        scale_by_inv<T>(s, elv, cols * chi_c, e->d_scal);
        log_s += std::log(nrm);
        trunc_den += tot;
        trunc_num += std::max(0.0, tot - kept2);
        e->spectra.zip[c] = sv;
        qa = qk;
        qnew[c + 1] = qk;
        Nvec[c] = N;
        abond[c + 1] = chi_c;
        ELvec[c + 1] = elv;
        EL[c + 1] = env_from_vectors(rowmem, elv, chi_c, st.bR, st.tp, st.nA[2], st.nW[2]);
        FP_CUDA(cudaStreamSynchronize(s));
        continue;
      }
      const int chi_c = (int)std::min<int64_t>({(int64_t)chi, rows, cols});
      const int k = prm.exact_svd ? (int)std::min(rows, cols)
                                  : (int)std::min<int64_t>({(int64_t)chi_c + prm.oversample, rows, cols});
      T* omega = ar.get_n<T>(cols * k);
      int64_t perm[2] = {st.bR, st.tp};
      gaussian_sketch<T>(s, omega, cols, k, cols, perm, e->cfg.seed, (uint64_t)e->layer, (uint64_t)c, w3);
      Env3 elc = EL[c];
      Lin A{rows, cols,
            [&](const T* X, T* Y, int64_t kk) { theta(st, elc, X, Y, kk); },
            [&](const T* Y, T* Z, int64_t kk) { theta_t(st, elc, Y, Z, kk); },
            // without a fit pass the zip-up's singular values set the row's scale
            [&](const T* Y, T* Z, int64_t kk) { apply(OP_THETA_T, st, elc, Y, Z, kk, prm.n_fit == 0); }};
      RsvdOut r = rsvd(ar, A, omega, k, prm.power_iters);
      // N = Q U[:, :chi_c]
      T* Ut = ar.get_n<T>((int64_t)k * k);
      convert_f64<T>(s, r.U, Ut, (int64_t)k * k);
      T* N = rowmem.get_n<T>(rows * chi_c);
      mm_right(rows, chi_c, k, r.Q, rows, Ut, k, N, rows, TALL_CALIBRATED);
      // sign gauge: weights from the sketch generator (stage 2) over the (a, Dn)
      // flat index; rows are stored Dn-major with a fastest
      double* sgn = ar.get_n<double>(chi_c);
      T* gw = ar.get_n<T>(rows);
      int64_t gperm[2] = {st.bD, a};
      gaussian_sketch<T>(s, gw, rows, 1, rows, gperm, e->cfg.seed, (uint64_t)e->layer, (uint64_t)c | (2ull << 16), w3);
      col_signs<T>(s, N, rows, chi_c, rows, gw, sgn);
      scale_cols<T>(s, N, rows, chi_c, rows, sgn);
      // EL_{c+1} vectors = Q_b W[:, :chi] diag(sigma * sign)
      double* sc = ar.get_n<double>(chi_c);
      double* sgd = ar.get_n<double>(chi_c);
      FP_CUDA(cudaMemcpyAsync(sgd, r.sigma.data(), sizeof(double) * chi_c, cudaMemcpyHostToDevice, s));
      mul_vec(s, sgd, sgn, sc, chi_c);
      T* elv = rowmem.get_n<T>(cols * chi_c);
      FP_CUDA(cudaMemcpyAsync(elv, r.QbW, sizeof(T) * cols * chi_c, cudaMemcpyDeviceToDevice, s));
      scale_cols<T>(s, elv, cols, chi_c, cols, sc);
      double nrm = host_norm(elv, cols * chi_c);
      FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "zip-up remainder vanished");
      scale_by_inv<T>(s, elv, cols * chi_c, e->d_scal);
      log_s += std::log(nrm);
      for (int j = 0; j < (int)r.sigma.size(); ++j) {
        double v2 = r.sigma[j] * r.sigma[j];
        trunc_den += v2;
        if (j >= chi_c) trunc_num += v2;
      }
      e->spectra.zip[c].assign(r.sigma.begin(), r.sigma.begin() + chi_c);
      Nvec[c] = N;
      abond[c + 1] = chi_c;
      ELvec[c + 1] = elv;
      EL[c + 1] = env_from_vectors(rowmem, elv, chi_c, st.bR, st.tp, st.nA[2], st.nW[2]);
      FP_CUDA(cudaStreamSynchronize(s));
    }
    // last site: Theta has a single column
    T* Nlast = nullptr;
    {
      Arena ar = arena();
      const int c = Ly - 1;
      Site st = make_site(ar, row, c, true, false);
      T* one = ar.get_n<T>(1);
      fill<T>(s, one, 1, T(1));
      const int64_t rows = (int64_t)EL[c].a * st.bD;
      T* yv = ar.get_n<T>(rows);
      apply(OP_THETA, st, EL[c], one, yv, 1, true);                  // [1][Dn][a]
      Nlast = rowmem.get_n<T>(rows);
      permute3<T>(s, yv, Nlast, 1, st.bD, EL[c].a, 0, 2, 1);        // -> [a][Dn][1]
      double nrm = host_norm(Nlast, rows);
      FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "zip-up last tensor vanished");
      scale_by_inv<T>(s, Nlast, rows, e->d_scal);
      log_s += std::log(nrm);
      FP_CUDA(cudaStreamSynchronize(s));
    }

    std::vector<void*> T_new(Ly, nullptr);
    std::vector<int> tb_new(Ly + 1, 1), ph_new(Ly, 1);
    for (int c = 0; c < Ly; ++c) ph_new[c] = bund(e->sites[e->layer][row * Ly + c], 3);
    double log_row = log_s;

    if (prm.n_fit == 0 || Ly == 1) {
      // boundary = zip-up isometries [a][Dn][chi] and the last tensor [a][Dn][1]
      for (int c = 0; c < Ly; ++c) {
        const int a = abond[c], b = (c < Ly - 1) ? abond[c + 1] : 1, Dn = ph_new[c];
        T* out = (T*)e->al.get(sizeof(T) * (int64_t)a * Dn * b);
        if (c < Ly - 1)
          permute3<T>(s, Nvec[c], out, b, Dn, a, 2, 1, 0);
        else
          FP_CUDA(cudaMemcpyAsync(out, Nlast, sizeof(T) * (int64_t)a * Dn, cudaMemcpyDeviceToDevice, s));
        T_new[c] = out;
        tb_new[c] = a;
        tb_new[c + 1] = b;
      }
    } else {
      if (sym) {
        if (prm.n_fit != 1) throw Error{FPEPS_ERR_UNSUPPORTED, "charge sectors: n_fit must be 0 or 1"};
        std::vector<std::vector<int32_t>> qfit;
        log_row = fit_sym(row, prm, Nvec, abond, EL, Nlast, T_new, tb_new, rowmem, qnew, qfit);
        qnew = qfit;
      } else {
        log_row = fit(row, prm, Nvec, abond, EL, Nlast, T_new, tb_new, rowmem, 1);
        // further passes start from the previous one, re-canonicalised left to right
        for (int pass = 2; pass <= prm.n_fit; ++pass) {
          Arena canon = arena();
          std::vector<T*> Nv2(Ly, nullptr);
          std::vector<int> ab2(Ly + 1, 1);
          std::vector<Env3> EL2(Ly);
          T* Nlast2 = nullptr;
          recanonicalize(row, T_new, tb_new, canon, Nv2, ab2, EL2, Nlast2);
          std::vector<void*> T_next(Ly, nullptr);
          std::vector<int> tb_next(Ly + 1, 1);
          log_row = fit(row, prm, Nv2, ab2, EL2, Nlast2, T_next, tb_next, canon, pass);
          for (void* p : T_new) e->al.put(p);
          T_new = T_next;
          tb_new = tb_next;
        }
      }
    }
    FP_CUDA(cudaStreamSynchronize(s));
    for (void* p : e->T) e->al.put(p);
    e->T = T_new;
    e->tb = tb_new;
    e->tphys = ph_new;
    e->log_scale += log_row;
    if (sym) e->qT = qnew;
    FP_CUDA(cudaEventRecord(ev1, s));
    FP_CUDA(cudaEventSynchronize(ev1));
    float ms = 0;
    FP_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (trace) {
      ph[5] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      fprintf(stderr, "[fpeps] row %d: total %.3f s  apply %.3f  qr %.3f  svd %.3f  (alg %.3e flop)\n", row, ph[5],
              ph[0], ph[1], ph[2], flops);
    }
    if (out) {
      out->seconds = ms * 1e-3;
      out->alg_flops = flops;
      out->log_scale = log_row;
      out->trunc_err_est = trunc_den > 0 ? trunc_num / trunc_den : 0.0;
    }
  }

  // Left-to-right gauge sweep of a fitted boundary F (F[0] unit norm, F[c > 0] right isometries
  // [a_{c-1}][Dn][a_c]) before another right-to-left fit pass, which needs the sites left of
  // each bond left-canonical: each site, with the triangular factor of the one before it
  // multiplied in, is split by a thin QR (Q the new left isometry, R carried right), and the
  // left environment of the next site is EL_{c+1} = (Theta_c^T N_c)^T, pattern 2(a) as in the
  // zip-up's remainder, normalised (the fit takes its scale from the first site, whose
  // environment is exactly 1). Output in the zip-up's form: Nvec[c] vectors [a_c][Dn][a_{c-1}],
  // abond, EL, and the unit-norm last tensor Nlast [a][Dn][1].
  void recanonicalize(int row, const std::vector<void*>& F, const std::vector<int>& tb, Arena& mem,
                      std::vector<T*>& Nvec, std::vector<int>& abond, std::vector<Env3>& EL, T*& Nlast) {
    fpeps_env* e = env;
    const int Ly = e->cfg.Ly;
    EL[0] = unit_env(mem);
    abond[0] = 1;
    Arena rmem = arena();
    T* Rt = nullptr;   // carried factor, a_in x a_in column-major (null: identity of size 1)
    for (int c = 0; c < Ly; ++c) {
      Arena ar = arena();
      const int a_in = tb[c], a_out = tb[c + 1];
      const int Dn = bund(e->sites[e->layer][row * Ly + c], 3);
      const int64_t m = (int64_t)a_in * Dn;
      // F_c [a_in][Dn][a_out] -> a_out vectors of (Dn, a_in), then X = R F_c on the a_in index
      T* Fv = ar.get_n<T>(m * a_out);
      permute3<T>(s, (const T*)F[c], Fv, a_in, Dn, a_out, 2, 1, 0);
      T* X = Fv;
      if (Rt) {
        X = ar.get_n<T>(m * a_out);
        mm(a_in, (int64_t)Dn * a_out, a_in, T(1), Rt, false, a_in, Fv, false, a_in, T(0), X, a_in);
      }
      if (c == Ly - 1) {   // the last tensor: X is [1][Dn][a] -> [a][Dn][1], unit norm
        Nlast = mem.get_n<T>(m);
        permute3<T>(s, X, Nlast, 1, Dn, a_in, 2, 1, 0);
        const double nrm = host_norm(Nlast, m);
        FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "re-canonicalisation: last tensor vanished");
        scale_by_inv<T>(s, Nlast, m, e->d_scal);
        abond[Ly - 1] = a_in;
        break;
      }
      T* Q = mem.get_n<T>(m * a_out);
      double* R = ar.get_n<double>((int64_t)a_out * a_out);
      qr(X, m, a_out, Q, R);
      Nvec[c] = Q;
      abond[c + 1] = a_out;
      // the factor for the next site (R row-major FP64 -> column-major copy)
      Arena rnew = arena();
      T* Rn = rnew.get_n<T>((int64_t)a_out * a_out);
      convert_f64_t<T>(s, R, a_out, a_out, Rn);
      rmem.reset();
      rmem.live = rnew.live;
      rnew.live.clear();
      Rt = Rn;
      // EL_{c+1}: Theta_c^T on the a_out columns of the isometry -> vectors [a_out][R][t']
      Site st = make_site(ar, row, c, true, false);
      const int64_t ncol = (int64_t)st.tp * st.bR;
      T* Z = ar.get_n<T>(ncol * a_out);
      theta_t(st, EL[c], Q, Z, a_out);
      const double nrm = host_norm(Z, ncol * a_out);
      FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "re-canonicalisation: left environment vanished");
      scale_by_inv<T>(s, Z, ncol * a_out, e->d_scal);
      EL[c + 1] = env_from_vectors(mem, Z, a_out, st.bR, st.tp, st.nA[2], st.nW[2]);
      FP_CUDA(cudaStreamSynchronize(s));
    }
  }

  // Right-to-left variational fit with controlled bond expansion (Fig. 3-5); pass p of the
  // row draws its CBE sketch at generator stage 1 + 16 (p - 1).
  double fit(int row, const fpeps_rsvd_params& prm, std::vector<T*>& Nvec, std::vector<int>& abond,
             std::vector<Env3>& EL, T* Nlast, std::vector<void*>& T_new, std::vector<int>& tb_new, Arena& rowmem,
             int pass) {
    fpeps_env* e = env;
    const int Ly = e->cfg.Ly;
    const int chi = e->cfg.chi;
    const int chi_t = prm.chi_tilde > 0 ? prm.chi_tilde : (chi + 9) / 10;
    const uint64_t w3 = (uint64_t)row | ((uint64_t)env->cur << 16);   // row | environment << 16
    // centre M [a_prev][Dn][a_c] as vectors (a_prev of them)
    Arena mmem = arena();
    int a_prev = abond[Ly - 1];
    int a_c = 1;
    const int64_t nlast = (int64_t)a_prev * bund(e->sites[e->layer][row * Ly + Ly - 1], 3);
    T* M = mmem.get_n<T>(nlast);
    FP_CUDA(cudaMemcpyAsync(M, Nlast, sizeof(T) * nlast, cudaMemcpyDeviceToDevice, s));
    // Nlast is [a][Dn][1] flat = vectors [a][Dn*1]: already "a_prev vectors of (Dn, a_c=1)"
    Arena ermem = arena();
    Env3 ER = unit_env(ermem);
    double rs = 0.0, rs_M = 0.0;
    for (int c = Ly - 1; c >= 1; --c) {
      Arena ar = arena();
      Site sc = make_site(ar, row, c, false, true);
      Site sl = make_site(ar, row, c - 1, true, false);
      const int Dn = sc.bD;
      const int64_t cols_a = (int64_t)Dn * a_c;
      // V^T = orth(M^T): (Dn a_c) x a_prev
      int a_eff;
      T* VT;
      if (a_prev >= cols_a) {
        a_eff = (int)cols_a;
        VT = ar.get_n<T>(cols_a * a_eff);
        set_identity<T>(s, VT, cols_a, a_eff);
      } else {
        a_eff = a_prev;
        VT = ar.get_n<T>(cols_a * a_eff);
        qr(M, cols_a, a_eff, VT, nullptr);
      }
      const int a2 = EL[c - 1].a;
      const int Dnl = sl.bD;
      const int64_t rows_a = (int64_t)a2 * Dnl;
      const int na = abond[c];          // columns of the zip-up isometry at c-1
      T* Nl = Nvec[c - 1];              // rows_a x na
      const int ct = (int)std::min<int64_t>({(int64_t)chi_t, rows_a - na, cols_a - a_eff});
      Env3 elc = EL[c - 1];
      Env3 erc = ER;
      T* Vp;
      int j;
      if (ct > 0) {
        const int k = (int)std::min<int64_t>({(int64_t)ct + prm.oversample, rows_a, cols_a});
        T* omega = ar.get_n<T>(cols_a * k);
        gaussian_sketch<T>(s, omega, cols_a, k, cols_a, nullptr, e->cfg.seed, (uint64_t)e->layer,
                           (uint64_t)c | ((uint64_t)(1 + 16 * (pass - 1)) << 16), w3);
        const int kmax = k;
        T* tmpA = ar.get_n<T>(std::max<int64_t>(a_eff, na) * kmax);
        T* Xp = ar.get_n<T>(std::max(cols_a, rows_a) * kmax);
        T* Zm = ar.get_n<T>(((int64_t)sl.tp * sl.bR) * kmax);
        Projector PR = projector(ar, VT, cols_a, a_eff);
        Projector PL = projector(ar, Nl, rows_a, na);
        auto projR = [&](const T* X, T* out, int64_t kk) { project_out(PR, X, out, kk, tmpA); };   // X - V^T (V X)
        auto projL = [&](T* Y, int64_t kk) { project_out(PL, Y, Y, kk, tmpA); };                 // Y - Nl (Nl^T Y)
        Lin A{rows_a, cols_a,
              [&](const T* X, T* Y, int64_t kk) {
                projR(X, Xp, kk);
                theta_r(sc, erc, Xp, Zm, kk);
                theta(sl, elc, Zm, Y, kk);
                projL(Y, kk);
              },
              [&](const T* Y, T* X, int64_t kk) {
                FP_CUDA(cudaMemcpyAsync(Xp, Y, sizeof(T) * rows_a * kk, cudaMemcpyDeviceToDevice, s));
                projL(Xp, kk);
                theta_t(sl, elc, Xp, Zm, kk);
                theta_r_t(sc, erc, Zm, X, kk);
                project_out(PR, X, X, kk, tmpA);   // X -= V^T (V X)
              }};
        RsvdOut r = rsvd(ar, A, omega, k, prm.power_iters);
        // right singular vectors of numerically zero singular values are not
        // determined by A: zero columns (sigma is sorted, so they are the last)
        {
          double tot = 0;
          for (double sv : r.sigma) tot += sv * sv;
          int live = 0;
          while (live < ct && r.sigma[live] * r.sigma[live] > 1e-30 * tot) ++live;
          if (live < ct) FP_CUDA(cudaMemsetAsync(r.QbW + cols_a * live, 0, sizeof(T) * cols_a * (ct - live), s));
        }
        // V' = orth([V^T | Vtil^T])
        j = a_eff + ct;
        T* cat = ar.get_n<T>(cols_a * j);
        copy_cols<T>(s, VT, cols_a, a_eff, cat);
        copy_cols<T>(s, r.QbW, cols_a, ct, cat + cols_a * a_eff);
        Vp = ar.get_n<T>(cols_a * j);
        qr(cat, cols_a, j, Vp, nullptr);
      } else {
        j = a_eff;
        Vp = VT;
      }
      // expanded right environment and the fitted tensor at c-1 (pattern 2(a))
      const int64_t nER = (int64_t)sl.tp * sl.bR;    // (t_{c-1}, L_c) space
      T* ERp = ar.get_n<T>(nER * j);
      apply(OP_THETA_R, sc, erc, Vp, ERp, j, true);
      T* Mp = ar.get_n<T>(rows_a * j);
      apply(OP_THETA, sl, elc, ERp, Mp, j, true);
      const int keep = (int)std::min<int64_t>({(int64_t)chi, rows_a, (int64_t)j});
      // SVD of M' = Q_m R_m,  R_m = U_r S W^T  (Jacobi on R_m^T: U_jac = W, V_jac = U_r)
      T* Qm = ar.get_n<T>(rows_a * j);
      double* Rm = ar.get_n<double>((int64_t)j * j);
      qr(Mp, rows_a, j, Qm, Rm);
      double* Uj = ar.get_n<double>((int64_t)j * j);
      double* Vj = ar.get_n<double>((int64_t)j * j);
      double* sg = ar.get_n<double>(j);
      int* order = ar.get_n<int>(j);
      {
        Phase ph_(this, 2);
        svd_jacobi_f64(s, Rm, j, Uj, sg, Vj, order, e->d_info, ar.get(64));
      }
      FP_CHECK(read_info() == 0, FPEPS_ERR_NUMERIC, "Jacobi SVD did not converge (fit)");
      double* Vs = ar.get_n<double>((int64_t)j * j);
      gather_cols_f64(s, Vj, order, j, Vs);
      T* Wt = ar.get_n<T>((int64_t)j * j);
      T* Urt = ar.get_n<T>((int64_t)j * j);
      convert_f64<T>(s, Uj, Wt, (int64_t)j * j);
      convert_f64<T>(s, Vs, Urt, (int64_t)j * j);
      // new right isometry N_c^T = V' W[:, :keep]  ->  [keep][Dn][a_c]
      T* Nc = (T*)e->al.get(sizeof(T) * cols_a * keep);
      mm_right(cols_a, keep, j, Vp, cols_a, Wt, j, Nc, cols_a, TALL_CALIBRATED);
      double* sgn = ar.get_n<double>(keep);
      T* gw = ar.get_n<T>(cols_a);
      gaussian_sketch<T>(s, gw, cols_a, 1, cols_a, nullptr, e->cfg.seed, (uint64_t)e->layer, (uint64_t)c | (2ull << 16),
                         w3);
      col_signs<T>(s, Nc, cols_a, keep, cols_a, gw, sgn);
      scale_cols<T>(s, Nc, cols_a, keep, cols_a, sgn);
      T_new[c] = Nc;
      tb_new[c] = keep;
      tb_new[c + 1] = a_c;
      // M_{c-1} = Q_m U_r[:, :keep] diag(S sign)  (vectors [keep][Dnl][a2]) -> [a2][Dnl][keep]
      double* scl = ar.get_n<double>(keep);
      mul_vec(s, sg, sgn, scl, keep);
      T* Mv = ar.get_n<T>(rows_a * keep);
      mm_right(rows_a, keep, j, Qm, rows_a, Urt, j, Mv, rows_a, TALL_CALIBRATED);
      scale_cols<T>(s, Mv, rows_a, keep, rows_a, scl);
      Arena mnew = arena();
      T* Mnext = mnew.get_n<T>(rows_a * keep);
      permute3<T>(s, Mv, Mnext, keep, Dnl, a2, 2, 1, 0);
      // ER_c vectors = ER' W[:, :keep] diag(sign)  -> [keep][L][t]
      T* erv = ar.get_n<T>(nER * keep);
      mm_right(nER, keep, j, ERp, nER, Wt, j, erv, nER, TALL_CALIBRATED);
      scale_cols<T>(s, erv, nER, keep, nER, sgn);
      double nrm = host_norm(erv, nER * keep);
      FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "right environment vanished");
      scale_by_inv<T>(s, erv, nER * keep, e->d_scal);
      rs_M = rs;
      rs += std::log(nrm);
      Arena ernew = arena();
      Env3 ERn = env_from_vectors(ernew, erv, keep, sl.bR, sl.tp, sl.nA[2], sl.nW[2]);
      {
        std::vector<double> sv(j);
        FP_CUDA(cudaMemcpyAsync(sv.data(), sg, sizeof(double) * j, cudaMemcpyDeviceToHost, s));
        FP_CUDA(cudaStreamSynchronize(s));
        e->spectra.fit[c - 1].assign(sv.begin(), sv.begin() + keep);
      }
      FP_CUDA(cudaStreamSynchronize(s));
      // rotate ownership
      ermem.reset();
      ermem.live = ernew.live;
      ernew.live.clear();
      ER = ERn;
      mmem.reset();
      mmem.live = mnew.live;
      mnew.live.clear();
      M = Mnext;
      a_c = keep;
      a_prev = a2;
    }
    // site 0: M_0 [1][Dn_0][a_0]
    const int Dn0 = bund(e->sites[e->layer][row * Ly], 3);
    const int64_t n0 = (int64_t)Dn0 * a_c;
    double nrm = host_norm(M, n0);
    FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "fit centre vanished");
    T* N0 = (T*)e->al.get(sizeof(T) * n0);
    FP_CUDA(cudaMemcpyAsync(N0, M, sizeof(T) * n0, cudaMemcpyDeviceToDevice, s));
    scale_by_inv<T>(s, N0, n0, e->d_scal);
    T_new[0] = N0;
    tb_new[0] = 1;
    tb_new[1] = a_c;
    FP_CUDA(cudaStreamSynchronize(s));
    return rs_M + std::log(nrm);
  }

  // ---------------------------------------------------------------- charge sectors: CBE fit
  using QKey = std::pair<int32_t, int32_t>;
  struct SecIdx {
    QKey q;
    std::vector<int64_t> ri, ci;
    int64_t *d_ri = nullptr, *d_ci = nullptr;
  };
  // charges shared by the rows and the columns (pairs per index), ascending, with
  // their index lists on the host and the device
  std::vector<SecIdx> sectors_of(Arena& ar, const std::vector<int32_t>& rowq, const std::vector<int32_t>& colq) {
    std::map<QKey, std::vector<int64_t>> rm, cm;
    for (int64_t i = 0; i < (int64_t)rowq.size() / 2; ++i) rm[{rowq[2 * i], rowq[2 * i + 1]}].push_back(i);
    for (int64_t i = 0; i < (int64_t)colq.size() / 2; ++i) cm[{colq[2 * i], colq[2 * i + 1]}].push_back(i);
    std::vector<SecIdx> out;
    for (auto& kv : rm) {
      auto it = cm.find(kv.first);
      if (it == cm.end()) continue;
      SecIdx x;
      x.q = kv.first;
      x.ri = kv.second;
      x.ci = it->second;
      out.push_back(std::move(x));
    }
    for (auto& x : out) {
      x.d_ri = ar.get_n<int64_t>((int64_t)x.ri.size());
      x.d_ci = ar.get_n<int64_t>((int64_t)x.ci.size());
      FP_CUDA(cudaMemcpyAsync(x.d_ri, x.ri.data(), sizeof(int64_t) * x.ri.size(), cudaMemcpyHostToDevice, s));
      FP_CUDA(cudaMemcpyAsync(x.d_ci, x.ci.data(), sizeof(int64_t) * x.ci.size(), cudaMemcpyHostToDevice, s));
    }
    return out;
  }
  struct Pick {
    double v;
    int n, j;
  };
  // the `keep` largest values over the sectors' offers (ties: sector, then index),
  // returned in sector order, then index
  static std::vector<Pick> pick_global(std::vector<Pick> cand, int keep) {
    std::sort(cand.begin(), cand.end(), [](const Pick& x, const Pick& y) {
      return x.v != y.v ? x.v < y.v : (x.n != y.n ? x.n < y.n : x.j < y.j);
    });
    cand.resize(std::min<size_t>(cand.size(), (size_t)std::max(keep, 0)));
    std::sort(cand.begin(), cand.end(), [](const Pick& x, const Pick& y) { return x.n != y.n ? x.n < y.n : x.j < y.j; });
    return cand;
  }

  // Right-to-left CBE fit with every factorisation split by the charge of the bond
  // a_{c-1} it straddles (the block-sparse form of fit(); see oracle/symmetric.py):
  // the CBE rSVD per sector (a sector offers at most min(chi_tilde, rows_Q - n_Q(a),
  // cols_Q - n_Q(V)) vectors; chi_tilde kept over all sectors), the SVD of the fitted
  // tensor per sector (chi kept over all sectors). qzip: charges of the zip-up bonds;
  // qout receives the charges of the fitted bonds.
  double fit_sym(int row, const fpeps_rsvd_params& prm, std::vector<T*>& Nvec, std::vector<int>& abond,
                 std::vector<Env3>& EL, T* Nlast, std::vector<void*>& T_new, std::vector<int>& tb_new, Arena& rowmem,
                 const std::vector<std::vector<int32_t>>& qzip, std::vector<std::vector<int32_t>>& qout) {
    (void)rowmem;
    fpeps_env* e = env;
    const int Ly = e->cfg.Ly;
    const int chi = e->cfg.chi;
    const int chi_t = prm.chi_tilde > 0 ? prm.chi_tilde : (chi + 9) / 10;
    const uint64_t w3 = (uint64_t)row | ((uint64_t)env->cur << 16);   // row | environment << 16
    Arena mmem = arena();
    int a_prev = abond[Ly - 1];
    int a_c = 1;
    const int64_t nlast = (int64_t)a_prev * bund(e->sites[e->layer][row * Ly + Ly - 1], 3);
    T* M = mmem.get_n<T>(nlast);
    FP_CUDA(cudaMemcpyAsync(M, Nlast, sizeof(T) * nlast, cudaMemcpyDeviceToDevice, s));
    Arena ermem = arena();
    Env3 ER = unit_env(ermem);
    double rs = 0.0, rs_M = 0.0;
    std::vector<int32_t> qright{0, 0};
    qout.assign(Ly + 1, std::vector<int32_t>{0, 0});
    for (int c = Ly - 1; c >= 1; --c) {
      Arena ar = arena();
      Site sc = make_site(ar, row, c, false, true);
      Site sl = make_site(ar, row, c - 1, true, false);
      const int Dn = sc.bD;
      const int64_t cols_a = (int64_t)Dn * a_c;
      const int a2 = EL[c - 1].a;
      const int Dnl = sl.bD;
      const int64_t rows_a = (int64_t)a2 * Dnl;
      const int na = abond[c];
      const std::vector<int32_t>& QD = e->sites[e->layer][row * Ly + c].qB[3];
      const std::vector<int32_t>& QDl = e->sites[e->layer][row * Ly + c - 1].qB[3];
      const std::vector<int32_t>& qa_prev = qzip[c];
      const std::vector<int32_t>& qa_left = qzip[c - 1];
      FP_CHECK((int64_t)QD.size() == 2 * (int64_t)Dn && (int64_t)qright.size() == 2 * (int64_t)a_c &&
                   (int64_t)qa_prev.size() == 2 * (int64_t)a_prev && a_prev == na &&
                   (int64_t)QDl.size() == 2 * (int64_t)Dnl && (int64_t)qa_left.size() == 2 * (int64_t)a2,
               FPEPS_ERR_STATE, "charge sectors: charge lists do not match the bonds (fit)");
      // columns (Dn_c, a_c), a_c fastest: Q_Dn + q_{a_c}; rows (Dn_{c-1}, a_{c-2}), a fastest: q_a - Q_Dn
      std::vector<int32_t> colq(2 * cols_a), rowq(2 * rows_a);
      for (int64_t d = 0; d < Dn; ++d)
        for (int64_t x = 0; x < a_c; ++x)
          for (int t = 0; t < 2; ++t) colq[2 * (d * a_c + x) + t] = QD[2 * d + t] + qright[2 * x + t];
      for (int64_t d = 0; d < Dnl; ++d)
        for (int64_t x = 0; x < a2; ++x)
          for (int t = 0; t < 2; ++t) rowq[2 * (d * a2 + x) + t] = qa_left[2 * x + t] - QDl[2 * d + t];
      // V^T = orth(M^T): rows of different sectors have disjoint supports, so the
      // orthonormalisation keeps every vector in its sector
      int a_eff;
      T* VT;
      std::vector<int32_t> qV;
      if (a_prev >= cols_a) {
        a_eff = (int)cols_a;
        VT = ar.get_n<T>(cols_a * a_eff);
        set_identity<T>(s, VT, cols_a, a_eff);
        qV = colq;
      } else {
        a_eff = a_prev;
        VT = ar.get_n<T>(cols_a * a_eff);
        qr(M, cols_a, a_eff, VT, nullptr);
        qV = qa_prev;
      }
      T* Nl = Nvec[c - 1];
      Env3 elc = EL[c - 1];
      Env3 erc = ER;
      // CBE: sector offers
      std::vector<SecIdx> cs = sectors_of(ar, rowq, colq);
      auto count_q = [](const std::vector<int32_t>& q, const QKey& k) {
        int64_t n = 0;
        for (size_t i = 0; i + 1 < q.size(); i += 2) n += (q[i] == k.first && q[i + 1] == k.second);
        return n;
      };
      std::vector<int64_t> capof(cs.size());
      int64_t capsum = 0;
      for (size_t n = 0; n < cs.size(); ++n) {
        capof[n] = std::min<int64_t>({(int64_t)chi_t, (int64_t)cs[n].ri.size() - count_q(qa_prev, cs[n].q),
                                      (int64_t)cs[n].ci.size() - count_q(qV, cs[n].q)});
        capsum += std::max<int64_t>(0, capof[n]);
      }
      const int ct = (int)std::min<int64_t>(chi_t, capsum);
      T* Vp;
      int j;
      std::vector<int32_t> qVp = qV;
      if (ct > 0) {
        std::vector<int> cap(cs.size()), kq(cs.size());
        int kmax = 0;
        for (size_t n = 0; n < cs.size(); ++n) {
          const int64_t rank = std::min<int64_t>((int64_t)cs[n].ri.size(), (int64_t)cs[n].ci.size());
          cap[n] = (int)std::max<int64_t>(0, std::min<int64_t>({(int64_t)ct, rank, capof[n]}));
          kq[n] = cap[n] > 0 ? (int)std::min<int64_t>((int64_t)cap[n] + prm.oversample, rank) : 0;
          kmax = std::max(kmax, kq[n]);
        }
        T* omega = ar.get_n<T>(cols_a * kmax);
        gaussian_sketch<T>(s, omega, cols_a, kmax, cols_a, nullptr, e->cfg.seed, (uint64_t)e->layer,
                           (uint64_t)c | (1ull << 16), w3);
        T* tmpA = ar.get_n<T>(std::max<int64_t>(a_eff, na) * kmax);
        T* Xp = ar.get_n<T>(std::max(cols_a, rows_a) * kmax);
        T* Zm = ar.get_n<T>(((int64_t)sl.tp * sl.bR) * kmax);
        T* fullc = ar.get_n<T>(cols_a * kmax);
        T* fullr = ar.get_n<T>(rows_a * kmax);
        Projector PR = projector(ar, VT, cols_a, a_eff);
        Projector PL = projector(ar, Nl, rows_a, na);
        auto a_fwd = [&](const T* X, T* Y, int64_t kk) {   // A = P_L^perp Theta2s P_R^perp
          project_out(PR, X, Xp, kk, tmpA);
          theta_r(sc, erc, Xp, Zm, kk);
          theta(sl, elc, Zm, Y, kk);
          project_out(PL, Y, Y, kk, tmpA);
        };
        auto a_bwd = [&](const T* Y, T* X, int64_t kk) {
          FP_CUDA(cudaMemcpyAsync(Xp, Y, sizeof(T) * rows_a * kk, cudaMemcpyDeviceToDevice, s));
          project_out(PL, Xp, Xp, kk, tmpA);
          theta_t(sl, elc, Xp, Zm, kk);
          theta_r_t(sc, erc, Zm, X, kk);
          project_out(PR, X, X, kk, tmpA);
        };
        std::vector<T*> rv(cs.size(), nullptr);
        std::vector<std::vector<double>> sig(cs.size());
        std::vector<Pick> cand;
        double tot = 0.0;
        for (size_t n = 0; n < cs.size(); ++n) {
          if (cap[n] == 0) continue;
          const int64_t nr = (int64_t)cs[n].ri.size(), nc = (int64_t)cs[n].ci.size();
          const int64_t* dri = cs[n].d_ri;
          const int64_t* dci = cs[n].d_ci;
          T* om = ar.get_n<T>(nc * kq[n]);
          gather_rows<T>(s, omega, cols_a, dci, nc, kq[n], om, nc);
          Lin A{nr, nc,
                [&, dri, dci, nr, nc](const T* X, T* Y, int64_t kk) {
                  FP_CUDA(cudaMemsetAsync(fullc, 0, sizeof(T) * cols_a * kk, s));
                  scatter_rows<T>(s, X, nc, dci, nc, kk, fullc, cols_a);
                  a_fwd(fullc, fullr, kk);
                  gather_rows<T>(s, fullr, rows_a, dri, nr, kk, Y, nr);
                },
                [&, dri, dci, nr, nc](const T* Y, T* Z, int64_t kk) {
                  FP_CUDA(cudaMemsetAsync(fullr, 0, sizeof(T) * rows_a * kk, s));
                  scatter_rows<T>(s, Y, nr, dri, nr, kk, fullr, rows_a);
                  a_bwd(fullr, fullc, kk);
                  gather_rows<T>(s, fullc, cols_a, dci, nc, kk, Z, nc);
                }};
          RsvdOut r = rsvd(ar, A, om, kq[n], prm.power_iters);
          rv[n] = r.QbW;
          sig[n] = r.sigma;
          for (double v : r.sigma) tot += v * v;
          for (int jj = 0; jj < cap[n]; ++jj) cand.push_back({-r.sigma[jj], (int)n, jj});
        }
        std::vector<Pick> kept = pick_global(cand, ct);
        j = a_eff + ct;
        T* cat = ar.get_n<T>(cols_a * j);
        FP_CUDA(cudaMemsetAsync(cat, 0, sizeof(T) * cols_a * j, s));
        copy_cols<T>(s, VT, cols_a, a_eff, cat);
        for (int m = 0; m < ct; ++m) {
          const SecIdx& x = cs[kept[m].n];
          const double v = sig[kept[m].n][kept[m].j];
          const int64_t nc = (int64_t)x.ci.size();
          if (tot > 0 && v * v > 1e-30 * tot)   // right vectors of null values are not determined: zero
            scatter_rows<T>(s, rv[kept[m].n] + (int64_t)kept[m].j * nc, nc, x.d_ci, nc, 1,
                            cat + cols_a * (int64_t)(a_eff + m), cols_a);
          qVp.push_back(x.q.first);
          qVp.push_back(x.q.second);
        }
        Vp = ar.get_n<T>(cols_a * j);
        qr(cat, cols_a, j, Vp, nullptr);
      } else {
        j = a_eff;
        Vp = VT;
      }
      // expanded right environment and the fitted tensor at c-1 (pattern 2(a))
      const int64_t nER = (int64_t)sl.tp * sl.bR;
      T* ERp = ar.get_n<T>(nER * j);
      apply(OP_THETA_R, sc, erc, Vp, ERp, j, true);
      T* Mp = ar.get_n<T>(rows_a * j);
      apply(OP_THETA, sl, elc, ERp, Mp, j, true);
      // SVD of M' per sector (rows: charge of a_{c-1} from the left, columns: of V')
      std::vector<SecIdx> ms = sectors_of(ar, rowq, qVp);
      std::vector<T*> Ls(ms.size()), Ws(ms.size());
      std::vector<std::vector<double>> sv(ms.size());
      std::vector<Pick> mc;
      double mtot = 0.0;
      int64_t rsum = 0;
      T* Bj = ar.get_n<T>(rows_a * j);
      for (size_t n = 0; n < ms.size(); ++n) {
        const int64_t nr = (int64_t)ms[n].ri.size(), ncj = (int64_t)ms[n].ci.size();
        const int rr = (int)std::min(nr, ncj);
        gather_rows<T>(s, Mp, rows_a, ms[n].d_ri, nr, j, Bj, nr);        // nr x j
        T* Bs = ar.get_n<T>(nr * ncj);
        for (int64_t q = 0; q < ncj; ++q)
          FP_CUDA(cudaMemcpyAsync(Bs + q * nr, Bj + ms[n].ci[q] * nr, sizeof(T) * nr, cudaMemcpyDeviceToDevice, s));
        const bool tall = nr >= ncj;
        const int64_t mm = tall ? nr : ncj;   // QR of the tall orientation
        T* Bt = Bs;
        if (!tall) {
          Bt = ar.get_n<T>(ncj * nr);
          transpose_block<T>(s, Bs, nr, nr, ncj, Bt, ncj);
        }
        T* Qm = ar.get_n<T>(mm * rr);
        double* Rm = ar.get_n<double>((int64_t)rr * rr);
        qr(Bt, mm, rr, Qm, Rm);
        double* Uj = ar.get_n<double>((int64_t)rr * rr);
        double* Vj = ar.get_n<double>((int64_t)rr * rr);
        double* sg = ar.get_n<double>(rr);
        int* order = ar.get_n<int>(rr);
        {
          Phase ph_(this, 2);
          svd_jacobi_f64(s, Rm, rr, Uj, sg, Vj, order, e->d_info, ar.get(64));
        }
        FP_CHECK(read_info() == 0, FPEPS_ERR_NUMERIC, "Jacobi SVD did not converge (sector fit)");
        double* Vs = ar.get_n<double>((int64_t)rr * rr);
        gather_cols_f64(s, Vj, order, rr, Vs);
        T* Wt = ar.get_n<T>((int64_t)rr * rr);
        T* Urt = ar.get_n<T>((int64_t)rr * rr);
        convert_f64<T>(s, Uj, Wt, (int64_t)rr * rr);
        convert_f64<T>(s, Vs, Urt, (int64_t)rr * rr);
        // tall: B = Q R, R = U_r S W^T -> left Q U_r (nr x rr), right W (ncj x rr);
        // wide: B^T = Q R likewise -> left W (nr x rr), right Q U_r (ncj x rr)
        T* QU = ar.get_n<T>(mm * rr);
        mm_right(mm, rr, rr, Qm, mm, Urt, rr, QU, mm, TALL_CALIBRATED);
        Ls[n] = tall ? QU : Wt;
        Ws[n] = tall ? Wt : QU;
        sv[n].resize(rr);
        FP_CUDA(cudaMemcpyAsync(sv[n].data(), sg, sizeof(double) * rr, cudaMemcpyDeviceToHost, s));
        FP_CUDA(cudaStreamSynchronize(s));
        for (int q = 0; q < rr; ++q) {
          mtot += sv[n][q] * sv[n][q];
          mc.push_back({-sv[n][q], (int)n, q});
        }
        rsum += rr;
      }
      const int keep = (int)std::min<int64_t>(chi, rsum);
      FP_CHECK(keep > 0, FPEPS_ERR_NUMERIC, "charge sectors: fitted tensor has no shared sector");
      std::vector<Pick> mk = pick_global(mc, keep);
      T* Wfull = ar.get_n<T>((int64_t)j * keep);
      T* Ufull = ar.get_n<T>(rows_a * keep);
      FP_CUDA(cudaMemsetAsync(Wfull, 0, sizeof(T) * j * keep, s));
      FP_CUDA(cudaMemsetAsync(Ufull, 0, sizeof(T) * rows_a * keep, s));
      std::vector<double> skeep(keep);
      std::vector<int32_t> qk(2 * (size_t)keep);
      for (int m = 0; m < keep; ++m) {
        const SecIdx& x = ms[mk[m].n];
        const int64_t nr = (int64_t)x.ri.size(), ncj = (int64_t)x.ci.size();
        const int q = mk[m].j;
        skeep[m] = sv[mk[m].n][q];
        if (mtot > 0 && skeep[m] * skeep[m] > 1e-30 * mtot)
          scatter_rows<T>(s, Ws[mk[m].n] + (int64_t)q * ncj, ncj, x.d_ci, ncj, 1, Wfull + (int64_t)m * j, j);
        scatter_rows<T>(s, Ls[mk[m].n] + (int64_t)q * nr, nr, x.d_ri, nr, 1, Ufull + (int64_t)m * rows_a, rows_a);
        qk[2 * m] = x.q.first;
        qk[2 * m + 1] = x.q.second;
      }
      // new right isometry N_c^T = V' W  ->  [keep][Dn][a_c]
      T* Nc = (T*)e->al.get(sizeof(T) * cols_a * keep);
      mm_right(cols_a, keep, j, Vp, cols_a, Wfull, j, Nc, cols_a, TALL_CUDA_CORES);
      double* sgn = ar.get_n<double>(keep);
      T* gw = ar.get_n<T>(cols_a);
      gaussian_sketch<T>(s, gw, cols_a, 1, cols_a, nullptr, e->cfg.seed, (uint64_t)e->layer, (uint64_t)c | (2ull << 16),
                         w3);
      col_signs<T>(s, Nc, cols_a, keep, cols_a, gw, sgn);
      scale_cols<T>(s, Nc, cols_a, keep, cols_a, sgn);
      T_new[c] = Nc;
      tb_new[c] = keep;
      tb_new[c + 1] = a_c;
      double* sgd = ar.get_n<double>(keep);
      FP_CUDA(cudaMemcpyAsync(sgd, skeep.data(), sizeof(double) * keep, cudaMemcpyHostToDevice, s));
      double* scl = ar.get_n<double>(keep);
      mul_vec(s, sgd, sgn, scl, keep);
      scale_cols<T>(s, Ufull, rows_a, keep, rows_a, scl);
      Arena mnew = arena();
      T* Mnext = mnew.get_n<T>(rows_a * keep);
      permute3<T>(s, Ufull, Mnext, keep, Dnl, a2, 2, 1, 0);
      T* erv = ar.get_n<T>(nER * keep);
      mm_right(nER, keep, j, ERp, nER, Wfull, j, erv, nER, TALL_CUDA_CORES);
      scale_cols<T>(s, erv, nER, keep, nER, sgn);
      double nrm = host_norm(erv, nER * keep);
      FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "right environment vanished");
      scale_by_inv<T>(s, erv, nER * keep, e->d_scal);
      rs_M = rs;
      rs += std::log(nrm);
      Arena ernew = arena();
      Env3 ERn = env_from_vectors(ernew, erv, keep, sl.bR, sl.tp, sl.nA[2], sl.nW[2]);
      e->spectra.fit[c - 1] = skeep;
      qright = qk;
      qout[c] = qk;
      FP_CUDA(cudaStreamSynchronize(s));
      ermem.reset();
      ermem.live = ernew.live;
      ernew.live.clear();
      ER = ERn;
      mmem.reset();
      mmem.live = mnew.live;
      mnew.live.clear();
      M = Mnext;
      a_c = keep;
      a_prev = a2;
    }
    const int Dn0 = bund(e->sites[e->layer][row * Ly], 3);
    const int64_t n0 = (int64_t)Dn0 * a_c;
    double nrm = host_norm(M, n0);
    FP_CHECK(nrm > 0, FPEPS_ERR_NUMERIC, "fit centre vanished");
    T* N0 = (T*)e->al.get(sizeof(T) * n0);
    FP_CUDA(cudaMemcpyAsync(N0, M, sizeof(T) * n0, cudaMemcpyDeviceToDevice, s));
    scale_by_inv<T>(s, N0, n0, e->d_scal);
    T_new[0] = N0;
    tb_new[0] = 1;
    tb_new[1] = a_c;
    FP_CUDA(cudaStreamSynchronize(s));
    return rs_M + std::log(nrm);
  }

  // ---------------------------------------------------------------- diagnostics
  // one site map of the staged row on host vectors (layouts in include/fpeps.h,
  // fpeps_apply_theta_op): the host arrays are brought to the layouts of theta,
  // theta_t, theta_r and theta_r_t, and the results back
  void apply_theta_host(fpeps_env* e, int op, int c, int a, const void* envh, int k, const void* in,
                        void* out) override {
    const int row = e->staged_row;
    FP_CHECK(row > 0, FPEPS_ERR_STATE, "no staged row");
    ensure_sandwich(e, e->layer, row);
    Arena ar = arena();
    const bool right = op >= 2;
    Site st = make_site(ar, row, c, !right, right);
    const int64_t t = st.t, L = st.bL, tp = st.tp, R = st.bR, Dn = st.bD;
    // environment: [a][t][L] (left) or [a][t'][R] (right); E bundle PEPO-outermost, Et [bond][bundle][a]
    const int64_t bond = right ? tp : t, bun = right ? R : L;
    T* ev = ar.get_n<T>((int64_t)a * bond * bun);
    FP_CUDA(cudaMemcpyAsync(ev, envh, sizeof(T) * a * bond * bun, cudaMemcpyHostToDevice, s));
    Env3 E;
    E.a = a;
    T* eo = ar.get_n<T>((int64_t)a * bond * bun);
    bundle_outer<T>(s, ev, eo, (int64_t)a * bond, st.nA[right ? 2 : 0], st.nW[right ? 2 : 0]);
    E.E = eo;
    T* et = ar.get_n<T>((int64_t)a * bond * bun);
    permute3<T>(s, ev, et, a, bond, bun, 1, 2, 0);
    E.Et = et;
    // sizes of the input and output per vector, and the host-side index pair to swap (0: none)
    int64_t n_in = 0, n_out = 0, in_d1 = 0, in_d2 = 0, out_d1 = 0, out_d2 = 0;
    switch (op) {
      case 0: n_in = tp * R; n_out = a * Dn; in_d1 = tp; in_d2 = R; out_d1 = Dn; out_d2 = a; break;
      case 1: n_in = a * Dn; n_out = tp * R; in_d1 = a; in_d2 = Dn; out_d1 = R; out_d2 = tp; break;
      case 2: n_in = Dn * a; n_out = t * L; out_d1 = L; out_d2 = t; break;
      default: n_in = t * L; n_out = Dn * a; in_d1 = t; in_d2 = L; break;
    }
    T* ih = ar.get_n<T>((int64_t)k * n_in);
    FP_CUDA(cudaMemcpyAsync(ih, in, sizeof(T) * k * n_in, cudaMemcpyHostToDevice, s));
    T* X = ih;
    if (in_d1) {
      X = ar.get_n<T>((int64_t)k * n_in);
      permute3<T>(s, ih, X, k, in_d1, in_d2, 0, 2, 1);
    }
    T* Y = ar.get_n<T>((int64_t)k * n_out);
    run_op(op, st, E, X, Y, k);
    T* oh = Y;
    if (out_d1) {
      oh = ar.get_n<T>((int64_t)k * n_out);
      permute3<T>(s, Y, oh, k, out_d1, out_d2, 0, 2, 1);
    }
    FP_CUDA(cudaMemcpyAsync(out, oh, sizeof(T) * k * n_out, cudaMemcpyDeviceToHost, s));
    FP_CUDA(cudaStreamSynchronize(s));
  }
};

EngineBase* make_engine(fpeps_env* env) {
  if (env->elem == 8) return new Engine<double>(env);
  return new Engine<float>(env);
}

}  // namespace fpeps
