// C ABI of libfpeps: environment lifecycle, the row state machine and
// checkpoints. Every entry point converts internal errors to fpeps_status.
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstring>
#include <exception>
#include <new>

#include "env.cuh"

using fpeps::Error;

namespace fpeps {

void* Allocator::get(size_t bytes) {
  void* p = nullptr;
  if (has) {
    p = a.alloc(a.ctx, bytes, (void*)stream);
    if (!p) throw Error{FPEPS_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes"};
    return p;
  }
  cudaError_t e = cudaMallocAsync(&p, bytes, stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    throw Error{FPEPS_ERR_OOM, "cudaMallocAsync failed for " + std::to_string(bytes) + " bytes"};
  }
  FP_CUDA(e);
  return p;
}

void Allocator::put(void* p) {
  if (!p) return;
  if (has) {
    a.free(a.ctx, p, (void*)stream);
    return;
  }
  cudaFreeAsync(p, stream);
}

// ------------------------------------------------------------------ accounting
namespace {
std::atomic<long long> g_launches{0};
std::mutex g_prof_mu;
bool g_prof_on = false;
struct ProfRec {
  cudaEvent_t e0, e1;
  double flops, bytes;
};
std::vector<ProfRec> g_prof[PROF_KINDS];
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ProfToken prof_begin(int kind, cudaStream_t s, double flops, double bytes) {
  ProfToken t;
  if (!g_prof_on) return t;
  t.kind = kind;
  t.flops = flops;
  t.bytes = bytes;
  FP_CUDA(cudaEventCreate(&t.e0));
  FP_CUDA(cudaEventRecord(t.e0, s));
  return t;
}

void prof_end(ProfToken& t, cudaStream_t s) {
  if (t.kind < 0) return;
  cudaEvent_t e1;
  FP_CUDA(cudaEventCreate(&e1));
  FP_CUDA(cudaEventRecord(e1, s));
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof[t.kind].push_back(ProfRec{t.e0, e1, t.flops, t.bytes});
  t.kind = -1;
}

namespace {

const int64_t kMagic = 0x3144425350455046LL;   // "FPEPSBD1"
const int64_t kQMagic = 0x3151425350455046LL;  // "FPEPSBQ1": optional bond-charge section

template <class F>
fpeps_status guard(fpeps_env* env, F&& f) {
  try {
    f();
    return FPEPS_OK;
  } catch (const Error& e) {
    if (env) {
      env->err = e.msg;
      if (e.st == FPEPS_ERR_CUDA) env->poisoned = true;
    }
    return e.st;
  } catch (const std::bad_alloc&) {
    if (env) env->err = "host allocation failed";
    return FPEPS_ERR_OOM;
  } catch (const std::exception& e) {
    if (env) env->err = e.what();
    return FPEPS_ERR_ARG;
  }
}

void site_dims(const fpeps_config& c, int r, int col, int D, int* d) {
  d[0] = col == 0 ? 1 : D;
  d[1] = r == 0 ? 1 : D;
  d[2] = col == c.Ly - 1 ? 1 : D;
  d[3] = r == c.Lx - 1 ? 1 : D;
}

void copy_convert(fpeps_env* env, const void* src, int src_f64, void* dst, size_t n) {
  cudaStream_t s = env->stream;
  const bool dst_f64 = env->elem == 8;
  if ((bool)src_f64 == dst_f64) {
    FP_CUDA(cudaMemcpyAsync(dst, src, n * env->elem, cudaMemcpyDeviceToDevice, s));
  } else if (src_f64) {
    fpeps::convert_f64<float>(s, (const double*)src, (float*)dst, (int64_t)n);
  } else {
    fpeps::to_f64<float>(s, (const float*)src, (double*)dst, (int64_t)n);
  }
}

void scan_channels(fpeps_env* env, int layer) {
  auto& sites = env->sites[layer];
  int maxch = 1;
  for (auto& h : sites) maxch = std::max(maxch, h.dW[0] * h.dW[1] * h.dW[2] * h.dW[3]);
  int* d_flags = (int*)env->al.get(sizeof(int) * maxch);
  std::vector<int> flags(maxch);
  for (auto& h : sites) {
    const int nch = h.dW[0] * h.dW[1] * h.dW[2] * h.dW[3];
    const char* W = (const char*)env->pepo[layer] + h.offW * env->elem;
    if (env->elem == 8)
      fpeps::pepo_scan<double>(env->stream, (const double*)W, h.dW, d_flags);
    else
      fpeps::pepo_scan<float>(env->stream, (const float*)W, h.dW, d_flags);
    FP_CUDA(cudaMemcpyAsync(flags.data(), d_flags, sizeof(int) * nch, cudaMemcpyDeviceToHost, env->stream));
    FP_CUDA(cudaStreamSynchronize(env->stream));
    h.ch.clear();
    for (int i = 0; i < nch; ++i) {
      if (!flags[i]) continue;
      int l = i / (h.dW[1] * h.dW[2] * h.dW[3]), u = (i / (h.dW[2] * h.dW[3])) % h.dW[1];
      int r = (i / h.dW[3]) % h.dW[2], d = i % h.dW[3];
      h.ch.insert(h.ch.end(), {l, u, r, d});
    }
  }
  env->al.put(d_flags);
}

void check_env(fpeps_env* env) {
  if (!env) throw Error{FPEPS_ERR_ARG, "env is NULL"};
  if (env->poisoned) throw Error{FPEPS_ERR_STATE, "env is poisoned by an earlier CUDA error: " + env->err};
}

void trivial_boundary(fpeps_env* env) {
  const int Ly = env->cfg.Ly;
  for (void* p : env->T) env->al.put(p);
  env->T.assign(Ly, nullptr);
  for (int c = 0; c < Ly; ++c) {
    env->T[c] = env->al.get(env->elem);
    if (env->elem == 8)
      fpeps::fill<double>(env->stream, (double*)env->T[c], 1, 1.0);
    else
      fpeps::fill<float>(env->stream, (float*)env->T[c], 1, 1.0f);
  }
  env->tb.assign(Ly + 1, 1);
  env->tphys.assign(Ly, 1);
}

void absorb(fpeps_env* env, int row, int layer) {
  const int Lx = env->cfg.Lx;
  if (layer != 0 && layer != 1) throw Error{FPEPS_ERR_ARG, "layer must be 0 or 1"};
  if (layer == 1 && !env->pepo[1]) throw Error{FPEPS_ERR_STATE, "env has no operator PEPO"};
  if (row < 0 || row >= Lx) throw Error{FPEPS_ERR_ARG, "row out of range"};
  if (row == 0) {
    env->layer = layer;
    env->log_scale = 0.0;
    env->have_value = false;
    env->state = fpeps::RowState::Ready;
    if (Lx == 1) {
      trivial_boundary(env);
      env->engine->close_row(env, 0);
      env->state = fpeps::RowState::Closed;
      env->next_row = 1;
      return;
    }
    env->engine->first_row(env, 0);
    env->next_row = 1;
    return;
  }
  if (env->state != fpeps::RowState::Ready || row != env->next_row || layer != env->layer)
    throw Error{FPEPS_ERR_STATE, "rows must be absorbed in order within one layer (expected row " +
                                     std::to_string(env->next_row) + ")"};
  if (row == Lx - 1) {
    env->engine->close_row(env, row);
    env->state = fpeps::RowState::Closed;
    env->next_row = Lx;
    return;
  }
  env->staged_row = row;
  env->state = fpeps::RowState::Staged;
}

fpeps_rsvd_params norm_params(const fpeps_rsvd_params* p) {
  if (!p) throw Error{FPEPS_ERR_ARG, "params is NULL"};
  fpeps_rsvd_params q = *p;
  if (q.oversample < 0 || q.power_iters < 0 || q.chi_tilde < 0) throw Error{FPEPS_ERR_ARG, "negative rSVD parameter"};
  if (q.n_fit < 0 || q.n_fit > FPEPS_MAX_FIT_PASSES) throw Error{FPEPS_ERR_UNSUPPORTED, "n_fit out of range"};
  return q;
}

void compress(fpeps_env* env, const fpeps_rsvd_params& prm, fpeps_stats* st) {
  if (env->state != fpeps::RowState::Staged) throw Error{FPEPS_ERR_STATE, "no interior row is staged"};
  env->engine->compress(env, env->staged_row, prm, st);
  env->next_row = env->staged_row + 1;
  env->state = fpeps::RowState::Ready;
}

void sweep(fpeps_env* env, int layer, const fpeps_rsvd_params& prm) {
  for (int r = 0; r < env->cfg.Lx; ++r) {
    absorb(env, r, layer);
    if (env->state == fpeps::RowState::Staged) compress(env, prm, nullptr);
  }
}

}  // namespace
}  // namespace fpeps

extern "C" {

fpeps_status fpeps_env_create(const fpeps_config* cfg, const void* peps_dev, const void* pepo_dev,
                              const int32_t* charges_host, int32_t dtype_in, void* cuda_stream,
                              const fpeps_allocator* alloc, fpeps_env** out) {
  if (!out || !cfg) return FPEPS_ERR_ARG;
  *out = nullptr;
  const fpeps_config c = *cfg;
  if (c.Lx < 1 || c.Ly < 1 || c.D < 1 || c.p < 1 || c.w < 1 || c.chi < 1 || !peps_dev) return FPEPS_ERR_ARG;
  if (c.prec < FPEPS_F64 || c.prec > FPEPS_BF16X3) return FPEPS_ERR_ARG;
  if (dtype_in != 0 && dtype_in != 1) return FPEPS_ERR_ARG;
  if (c.Ly > 4096 || c.Lx > 4096 || c.D > 64 || c.p > 64 || c.w > 64) return FPEPS_ERR_ARG;
  if (c.n_envs < 1 || c.n_envs > FPEPS_MAX_ENVS) return FPEPS_ERR_ARG;
  if (c.symmetry != 0 && c.symmetry != 1) return FPEPS_ERR_ARG;
  if ((c.symmetry == 1) != (charges_host != nullptr)) return FPEPS_ERR_ARG;
  fpeps_env* env = new (std::nothrow) fpeps_env();
  if (!env) return FPEPS_ERR_OOM;
  env->cfg = c;
  env->slots.resize((size_t)c.n_envs);
  env->cur = 0;
  env->elem = c.prec == FPEPS_F64 ? 8 : 4;
  env->stream = (cudaStream_t)cuda_stream;
  env->al.stream = env->stream;
  if (alloc && alloc->alloc && alloc->free) {
    env->al.a = *alloc;
    env->al.has = true;
  }
  fpeps_status st = fpeps::guard(env, [&] {
    // site dimensions and packed offsets
    size_t offA = 0, offW = 0, offI = 0;
    for (int layer = 0; layer < 2; ++layer) env->sites[layer].resize((size_t)c.Lx * c.Ly);
    for (int r = 0; r < c.Lx; ++r)
      for (int col = 0; col < c.Ly; ++col) {
        const size_t i = (size_t)r * c.Ly + col;
        int dA[4], dW[4];
        fpeps::site_dims(c, r, col, c.D, dA);
        fpeps::site_dims(c, r, col, c.w, dW);
        auto& h0 = env->sites[0][i];
        auto& h1 = env->sites[1][i];
        for (int q = 0; q < 4; ++q) { h0.dA[q] = h1.dA[q] = dA[q]; h0.dW[q] = 1; h1.dW[q] = dW[q]; }
        h0.dA[4] = h1.dA[4] = c.p;
        h0.dW[4] = h0.dW[5] = h1.dW[4] = h1.dW[5] = c.p;
        h0.offA = h1.offA = offA;
        offA += (size_t)dA[0] * dA[1] * dA[2] * dA[3] * c.p;
        h1.offW = offW;
        offW += (size_t)dW[0] * dW[1] * dW[2] * dW[3] * c.p * c.p;
        h0.offW = offI;
        offI += (size_t)c.p * c.p;
      }
    if (c.symmetry == 1) {
      // leg charges -> bundle charges Q = q_ket - q_pepo - q_bra per (ket, PEPO, bra)
      // bundle index, bra fastest; the identity PEPO of layer 0 carries no charge
      const size_t n = (size_t)c.Lx * c.Ly;
      const int32_t* q = charges_host;
      std::vector<const int32_t*> qa(n * 4), qw(n * 4, nullptr);
      for (size_t i = 0; i < n; ++i)
        for (int l = 0; l < 4; ++l) {
          qa[i * 4 + l] = q;
          q += 2 * env->sites[1][i].dA[l];
        }
      if (pepo_dev)
        for (size_t i = 0; i < n; ++i)
          for (int l = 0; l < 4; ++l) {
            qw[i * 4 + l] = q;
            q += 2 * env->sites[1][i].dW[l];
          }
      for (int layer = 0; layer < 2; ++layer)
        for (size_t i = 0; i < n; ++i) {
          auto& h = env->sites[layer][i];
          for (int l = 0; l < 4; ++l) {
            const int dk = h.dA[l], dw = h.dW[l];
            const int32_t* qk = qa[i * 4 + l];
            const int32_t* qp = layer == 1 ? qw[i * 4 + l] : nullptr;
            std::vector<int32_t> v((size_t)2 * dk * dw * dk);
            for (int x = 0; x < dk; ++x)
              for (int y = 0; y < dw; ++y)
                for (int z = 0; z < dk; ++z)
                  for (int t = 0; t < 2; ++t)
                    v[2 * (((size_t)x * dw + y) * dk + z) + t] = qk[2 * x + t] - (qp ? qp[2 * y + t] : 0) - qk[2 * z + t];
            h.qB[l] = std::move(v);
          }
        }
    }
    FP_CUDA(cudaMallocHost((void**)&env->h_info, 16 * sizeof(int)));
    FP_CUDA(cudaMallocHost((void**)&env->h_scal, 16 * sizeof(double)));
    env->d_info = (int*)env->al.get(16 * sizeof(int));
    env->d_scal = (double*)env->al.get(16 * sizeof(double));
    env->peps = env->al.get(offA * env->elem);
    fpeps::copy_convert(env, peps_dev, dtype_in == 0, env->peps, offA);
    if (pepo_dev) {
      env->pepo[1] = env->al.get(offW * env->elem);
      fpeps::copy_convert(env, pepo_dev, dtype_in == 0, env->pepo[1], offW);
    }
    // identity PEPO: W[0,0,0,0,p,p'] = delta
    std::vector<double> eye((size_t)c.p * c.p, 0.0);
    for (int q = 0; q < c.p; ++q) eye[(size_t)q * c.p + q] = 1.0;
    std::vector<double> idall(offI);
    for (size_t i = 0; i < offI; i += eye.size()) std::memcpy(&idall[i], eye.data(), eye.size() * sizeof(double));
    void* tmp = env->al.get(offI * sizeof(double));
    FP_CUDA(cudaMemcpyAsync(tmp, idall.data(), offI * sizeof(double), cudaMemcpyHostToDevice, env->stream));
    env->pepo[0] = env->al.get(offI * env->elem);
    fpeps::copy_convert(env, tmp, 1, env->pepo[0], offI);
    FP_CUDA(cudaStreamSynchronize(env->stream));
    env->al.put(tmp);
    fpeps::scan_channels(env, 0);
    if (pepo_dev) fpeps::scan_channels(env, 1);
    env->engine = fpeps::make_engine(env);
    FP_CUDA(cudaStreamSynchronize(env->stream));
  });
  if (st != FPEPS_OK) {
    fpeps_env_destroy(env);
    return st;
  }
  *out = env;
  return FPEPS_OK;
}

fpeps_status fpeps_absorb_row(fpeps_env* env, int32_t row, int32_t layer) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    fpeps::absorb(env, row, layer);
  });
}

fpeps_status fpeps_compress_rsvd(fpeps_env* env, const fpeps_rsvd_params* params, fpeps_stats* out_host) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    fpeps_rsvd_params p = fpeps::norm_params(params);
    fpeps::compress(env, p, out_host);
  });
}

fpeps_status fpeps_sweep_value(fpeps_env* env, double* log_abs, int32_t* sign) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (!log_abs || !sign) throw Error{FPEPS_ERR_ARG, "NULL output"};
    if (!env->have_value) throw Error{FPEPS_ERR_STATE, "no closed sweep"};
    *log_abs = env->value_log;
    *sign = env->value_sign;
  });
}

fpeps_status fpeps_contract_norm(fpeps_env* env, const fpeps_rsvd_params* params, double* log_abs, int32_t* sign) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (!log_abs || !sign) throw Error{FPEPS_ERR_ARG, "NULL output"};
    fpeps_rsvd_params p = fpeps::norm_params(params);
    fpeps::sweep(env, 0, p);
    *log_abs = env->value_log;
    *sign = env->value_sign;
  });
}

fpeps_status fpeps_expect(fpeps_env* env, const fpeps_rsvd_params* params, double* value, double* log_abs_num,
                          int32_t* sign_num) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (!value) throw Error{FPEPS_ERR_ARG, "NULL output"};
    if (!env->pepo[1]) throw Error{FPEPS_ERR_STATE, "env has no operator PEPO"};
    fpeps_rsvd_params p = fpeps::norm_params(params);
    fpeps::sweep(env, 1, p);
    const double ln = env->value_log;
    const int sn = env->value_sign;
    fpeps::sweep(env, 0, p);
    *value = sn * env->value_sign * std::exp(ln - env->value_log);
    if (log_abs_num) *log_abs_num = ln;
    if (sign_num) *sign_num = sn;
  });
}

fpeps_status fpeps_export_boundary(fpeps_env* env, void* host_buf, size_t* bytes) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (!bytes) throw Error{FPEPS_ERR_ARG, "bytes is NULL"};
    if (env->T.empty() || env->state == fpeps::RowState::Closed)
      throw Error{FPEPS_ERR_STATE, "no boundary to export"};
    const int Ly = env->cfg.Ly;
    size_t head = sizeof(int64_t) * (5 + (Ly + 1) + Ly) + sizeof(double);
    size_t total = head;
    std::vector<size_t> n(Ly);
    for (int c = 0; c < Ly; ++c) {
      n[c] = (size_t)env->tb[c] * env->tphys[c] * env->tb[c + 1];
      total += n[c] * env->elem;
    }
    // charge-sector mode: the bonds' charge pairs follow the tensors
    const bool with_q = (int)env->qT.size() == Ly + 1;
    const size_t tensors_end = total;
    size_t nq = 0;
    if (with_q) {
      for (int c = 0; c <= Ly; ++c) {
        if ((int64_t)env->qT[c].size() != 2 * (int64_t)env->tb[c]) throw Error{FPEPS_ERR_STATE, "bond charges out of step"};
        nq += env->qT[c].size();
      }
      total += sizeof(int64_t) + ((nq * sizeof(int32_t) + 7) & ~(size_t)7);
    }
    if (!host_buf) {
      *bytes = total;
      return;
    }
    if (*bytes < total) throw Error{FPEPS_ERR_ARG, "buffer too small"};
    char* p = (char*)host_buf;
    int64_t* h = (int64_t*)p;
    h[0] = fpeps::kMagic; h[1] = Ly; h[2] = env->next_row; h[3] = env->layer; h[4] = env->elem;
    for (int c = 0; c <= Ly; ++c) h[5 + c] = env->tb[c];
    for (int c = 0; c < Ly; ++c) h[5 + Ly + 1 + c] = env->tphys[c];
    std::memcpy(p + head - sizeof(double), &env->log_scale, sizeof(double));
    size_t off = head;
    for (int c = 0; c < Ly; ++c) {
      FP_CUDA(cudaMemcpyAsync(p + off, env->T[c], n[c] * env->elem, cudaMemcpyDeviceToHost, env->stream));
      off += n[c] * env->elem;
    }
    if (with_q) {
      std::memcpy(p + tensors_end, &fpeps::kQMagic, sizeof(int64_t));
      int32_t* q = (int32_t*)(p + tensors_end + sizeof(int64_t));
      for (int c = 0; c <= Ly; ++c) {
        std::memcpy(q, env->qT[c].data(), env->qT[c].size() * sizeof(int32_t));
        q += env->qT[c].size();
      }
      std::memset(q, 0, (char*)(p + total) - (char*)q);
    }
    FP_CUDA(cudaStreamSynchronize(env->stream));
    *bytes = total;
  });
}

fpeps_status fpeps_import_boundary(fpeps_env* env, const void* host_buf, size_t bytes, int32_t next_row,
                                   int32_t layer) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (!host_buf) throw Error{FPEPS_ERR_ARG, "NULL buffer"};
    const int Ly = env->cfg.Ly;
    size_t head = sizeof(int64_t) * (5 + (Ly + 1) + Ly) + sizeof(double);
    if (bytes < head) throw Error{FPEPS_ERR_ARG, "buffer too small"};
    // the checkpoint may live in host or in device memory
    cudaPointerAttributes pa;
    bool on_dev = cudaPointerGetAttributes(&pa, host_buf) == cudaSuccess && pa.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    std::vector<char> hcopy;
    const char* src = (const char*)host_buf;
    if (on_dev) {
      hcopy.resize(head);
      FP_CUDA(cudaMemcpyAsync(hcopy.data(), host_buf, head, cudaMemcpyDeviceToHost, env->stream));
      FP_CUDA(cudaStreamSynchronize(env->stream));
    }
    const char* p = on_dev ? hcopy.data() : src;
    const int64_t* h = (const int64_t*)p;
    if (h[0] != fpeps::kMagic || h[1] != Ly || h[4] != env->elem) throw Error{FPEPS_ERR_ARG, "bad checkpoint header"};
    if (next_row < 1 || next_row >= env->cfg.Lx) throw Error{FPEPS_ERR_ARG, "next_row out of range"};
    if (layer != 0 && layer != 1) throw Error{FPEPS_ERR_ARG, "bad layer"};
    if (layer == 1 && !env->pepo[1]) throw Error{FPEPS_ERR_STATE, "env has no operator PEPO"};
    std::vector<int> tb(Ly + 1), ph(Ly);
    for (int c = 0; c <= Ly; ++c) tb[c] = (int)h[5 + c];
    for (int c = 0; c < Ly; ++c) ph[c] = (int)h[5 + Ly + 1 + c];
    if (tb[0] != 1 || tb[Ly] != 1) throw Error{FPEPS_ERR_ARG, "boundary end bonds must be 1"};
    size_t total = head;
    for (int c = 0; c < Ly; ++c) {
      if (tb[c] < 1 || ph[c] < 1) throw Error{FPEPS_ERR_ARG, "bad boundary dims"};
      total += (size_t)tb[c] * ph[c] * tb[c + 1] * env->elem;
    }
    if (bytes < total) throw Error{FPEPS_ERR_ARG, "buffer shorter than its header says"};
    // optional bond charges after the tensors (charge-sector mode)
    std::vector<std::vector<int32_t>> qT;
    if (bytes >= total + sizeof(int64_t)) {
      size_t nq = 0;
      for (int c = 0; c <= Ly; ++c) nq += 2 * (size_t)tb[c];
      std::vector<char> tail(bytes - total);
      if (on_dev) {
        FP_CUDA(cudaMemcpyAsync(tail.data(), src + total, tail.size(), cudaMemcpyDeviceToHost, env->stream));
        FP_CUDA(cudaStreamSynchronize(env->stream));
      } else {
        std::memcpy(tail.data(), src + total, tail.size());
      }
      int64_t qm = 0;
      std::memcpy(&qm, tail.data(), sizeof(int64_t));
      if (qm != fpeps::kQMagic) throw Error{FPEPS_ERR_ARG, "unknown data after the boundary tensors"};
      if (env->cfg.symmetry != 1) throw Error{FPEPS_ERR_ARG, "bond charges given to an env without charge sectors"};
      if (tail.size() < sizeof(int64_t) + nq * sizeof(int32_t)) throw Error{FPEPS_ERR_ARG, "bond charges truncated"};
      const int32_t* q = (const int32_t*)(tail.data() + sizeof(int64_t));
      qT.assign(Ly + 1, {});
      for (int c = 0; c <= Ly; ++c) {
        qT[c].assign(q, q + 2 * tb[c]);
        q += 2 * tb[c];
      }
    }
    for (void* q : env->T) env->al.put(q);
    env->T.assign(Ly, nullptr);
    size_t off = head;
    for (int c = 0; c < Ly; ++c) {
      size_t nb = (size_t)tb[c] * ph[c] * tb[c + 1] * env->elem;
      env->T[c] = env->al.get(nb);
      FP_CUDA(cudaMemcpyAsync(env->T[c], src + off, nb, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              env->stream));
      off += nb;
    }
    std::memcpy(&env->log_scale, p + head - sizeof(double), sizeof(double));
    if (!on_dev) FP_CUDA(cudaStreamSynchronize(env->stream));
    env->tb = tb;
    env->tphys = ph;
    env->qT = qT;      // empty unless the checkpoint carries bond charges
    env->layer = layer;
    env->next_row = next_row;
    env->state = fpeps::RowState::Ready;
    env->have_value = false;
  });
}

const char* fpeps_last_error(const fpeps_env* env) { return env ? env->err.c_str() : "env is NULL"; }

fpeps_status fpeps_env_select(fpeps_env* env, int32_t e) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (e < 0 || e >= (int32_t)env->slots.size()) throw Error{FPEPS_ERR_ARG, "environment index out of range"};
    if (e == env->cur) return;
    // park the selected environment's state, bring in environment e's
    fpeps_env::Slot& out = env->slots[env->cur];
    out.T.swap(env->T);
    out.tb.swap(env->tb);
    out.tphys.swap(env->tphys);
    out.qT.swap(env->qT);
    out.log_scale = env->log_scale;
    out.next_row = env->next_row;
    out.layer = env->layer;
    out.state = env->state;
    out.staged_row = env->staged_row;
    out.have_value = env->have_value;
    out.value_log = env->value_log;
    out.value_sign = env->value_sign;
    std::swap(out.spectra, env->spectra);
    fpeps_env::Slot& in = env->slots[e];
    env->T.swap(in.T);
    env->tb.swap(in.tb);
    env->tphys.swap(in.tphys);
    env->qT.swap(in.qT);
    env->log_scale = in.log_scale;
    env->next_row = in.next_row;
    env->layer = in.layer;
    env->state = in.state;
    env->staged_row = in.staged_row;
    env->have_value = in.have_value;
    env->value_log = in.value_log;
    env->value_sign = in.value_sign;
    std::swap(env->spectra, in.spectra);
    in = fpeps_env::Slot{};
    env->cur = e;
  });
}

void fpeps_env_destroy(fpeps_env* env) {
  if (!env) return;
  try {
    if (env->engine) delete env->engine;
    env->engine = nullptr;
    for (int layer = 0; layer < 2; ++layer)
      for (auto& sd : env->sand[layer])
        for (void* b : sd.bufs) env->al.put(b);
    for (void* p : env->T) env->al.put(p);
    for (size_t i = 0; i < env->slots.size(); ++i)
      if ((int)i != env->cur)
        for (void* p : env->slots[i].T) env->al.put(p);
    env->al.put(env->peps);
    env->al.put(env->pepo[0]);
    env->al.put(env->pepo[1]);
    env->al.put(env->d_info);
    env->al.put(env->d_scal);
    if (env->stream || !env->al.has) cudaStreamSynchronize(env->stream);
    if (env->h_info) cudaFreeHost(env->h_info);
    if (env->h_scal) cudaFreeHost(env->h_scal);
  } catch (...) {
  }
  delete env;
}

fpeps_status fpeps_boundary_shape(const fpeps_env* env, int32_t c, int32_t* t_left, int32_t* phys, int32_t* t_right) {
  if (!env || !t_left || !phys || !t_right) return FPEPS_ERR_ARG;
  if (c < 0 || c >= (int)env->tphys.size()) return FPEPS_ERR_ARG;
  *t_left = env->tb[c];
  *phys = env->tphys[c];
  *t_right = env->tb[c + 1];
  return FPEPS_OK;
}

fpeps_status fpeps_bond_spectrum(const fpeps_env* env, int32_t which, int32_t c, double* sv_host, int32_t* n_inout) {
  if (!env || !n_inout || (which != 0 && which != 1)) return FPEPS_ERR_ARG;
  const auto& v = which == 0 ? env->spectra.zip : env->spectra.fit;
  if (c < 0 || c >= (int)v.size()) return FPEPS_ERR_ARG;
  const auto& s = v[c];
  int n = (int)s.size();
  if (sv_host) {
    int m = std::min(n, *n_inout);
    std::memcpy(sv_host, s.data(), sizeof(double) * m);
  }
  *n_inout = n;
  return FPEPS_OK;
}

fpeps_status fpeps_apply_theta(fpeps_env* env, int32_t c, int32_t a, const void* el_host, int32_t k,
                               const void* x_host, void* y_host) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (env->state != fpeps::RowState::Staged) throw Error{FPEPS_ERR_STATE, "no staged row"};
    if (c < 0 || c >= env->cfg.Ly || a < 1 || k < 1 || !el_host || !x_host || !y_host)
      throw Error{FPEPS_ERR_ARG, "bad argument"};
    env->engine->apply_theta_host(env, 0, c, a, el_host, k, x_host, y_host);
  });
}

fpeps_status fpeps_apply_theta_op(fpeps_env* env, int32_t op, int32_t c, int32_t a, const void* env_host, int32_t k,
                                  const void* in_host, void* out_host) {
  return fpeps::guard(env, [&] {
    fpeps::check_env(env);
    if (op < 0 || op > 3 || c < 0 || c >= env->cfg.Ly || a < 1 || k < 1 || !env_host || !in_host || !out_host)
      throw Error{FPEPS_ERR_ARG, "bad argument"};
    if (env->state != fpeps::RowState::Staged) throw Error{FPEPS_ERR_STATE, "no staged row"};
    env->engine->apply_theta_host(env, op, c, a, env_host, k, in_host, out_host);
  });
}

fpeps_status fpeps_selftest_wait_timeout(void* cuda_stream) {
  return fpeps::guard(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // a 128-row product runs on a single CTA, a 256-row one on a CTA pair
    int timed_out = 0;
    for (const int64_t M : {128, 256}) {
      const int64_t N = 128, K = 32;
      float *A = nullptr, *B = nullptr, *C = nullptr;
      const size_t sb = fpeps::gemm_tc_scratch_bytes(FPEPS_TF32X3, M, N, K);
      int* err = nullptr;
      FP_CUDA(cudaMallocAsync((void**)&A, sizeof(float) * M * K, s));
      FP_CUDA(cudaMallocAsync((void**)&B, sizeof(float) * N * K, s));
      FP_CUDA(cudaMallocAsync((void**)&C, sizeof(float) * M * N, s));
      FP_CUDA(cudaMallocAsync((void**)&err, sb, s));
      FP_CUDA(cudaMemsetAsync(A, 0, sizeof(float) * M * K, s));
      FP_CUDA(cudaMemsetAsync(B, 0, sizeof(float) * N * K, s));
      FP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
      fpeps::gemm_tc(s, FPEPS_TF32X3, M, N, K, A, K, B, K, C, fpeps::out_rowmajor(M, N, N), err, sb, true);
      int h = 0;
      FP_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
      FP_CUDA(cudaStreamSynchronize(s));
      cudaFreeAsync(A, s);
      cudaFreeAsync(B, s);
      cudaFreeAsync(C, s);
      cudaFreeAsync(err, s);
      FP_CUDA(cudaStreamSynchronize(s));
      timed_out += h != 0;
    }
    if (timed_out == 2) throw Error{FPEPS_ERR_TIMEOUT, "tensor-core GEMM: bounded waits ran out as designed"};
  });
}

fpeps_status fpeps_gemm_f32(int32_t mode, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                            const float* B, int64_t ldb, float* C, void* cuda_stream) {
  return fpeps::guard(nullptr, [&] {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || lda < K || ldb < K) throw Error{FPEPS_ERR_ARG, "bad GEMM"};
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const fpeps::OutMap om = fpeps::out_rowmajor(M, N, N);
    if (mode == FPEPS_F32) {
      fpeps::gemm_simt<float>(s, M, N, K, 1.0f, A, lda, 1, B, ldb, 1, 0.0f, C, om);
      return;
    }
    if (mode != FPEPS_TF32X3 && mode != FPEPS_BF16X3) throw Error{FPEPS_ERR_UNSUPPORTED, "mode"};
    if (!fpeps::gemm_tc_supported(M, N, K, lda, ldb) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
      throw Error{FPEPS_ERR_UNSUPPORTED, "shape not supported by the tensor-core kernel"};
    const size_t sb = fpeps::gemm_tc_scratch_bytes(mode, M, N, K);
    int* err = nullptr;
    FP_CUDA(cudaMallocAsync((void**)&err, sb, s));
    FP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    fpeps::gemm_tc(s, mode, M, N, K, A, lda, B, ldb, C, om, err, sb);
    int h = 0;
    FP_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FP_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(err, s);
    if (h) throw Error{FPEPS_ERR_TIMEOUT, "tensor-core GEMM timed out"};
  });
}

fpeps_status fpeps_svd_f64(const double* M, int32_t k, double* U, double* sigma, double* V, void* cuda_stream) {
  return fpeps::guard(nullptr, [&] {
    if (!M || !U || !sigma || !V || k < 1 || k > 1024) throw Error{FPEPS_ERR_ARG, "bad SVD arguments"};
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t kk = (size_t)k * k;
    char* scr = nullptr;
    const size_t bytes = 2 * kk * sizeof(double) + ((size_t)k * sizeof(int) + 255) / 256 * 256 + 256;
    FP_CUDA(cudaMallocAsync((void**)&scr, bytes, s));
    double* Mw = (double*)scr;
    double* Vw = Mw + kk;
    int* order = (int*)(Vw + kk);
    void* ws = scr + bytes - 256;
    int* info = (int*)ws + 32;
    FP_CUDA(cudaMemcpyAsync(Mw, M, kk * sizeof(double), cudaMemcpyDeviceToDevice, s));
    fpeps::svd_jacobi_f64(s, Mw, k, U, sigma, Vw, order, info, ws);
    fpeps::gather_cols_f64(s, Vw, order, k, V);
    FP_CUDA(cudaFreeAsync(scr, s));
    FP_CUDA(cudaStreamSynchronize(s));
  });
}

int64_t fpeps_launch_count(void) { return fpeps::g_launches.load(); }

fpeps_status fpeps_profile(int32_t enable) {
  std::lock_guard<std::mutex> lk(fpeps::g_prof_mu);
  for (auto& v : fpeps::g_prof)
    for (auto& r : v) {
      cudaEventDestroy(r.e0);
      cudaEventDestroy(r.e1);
    }
  for (auto& v : fpeps::g_prof) v.clear();
  fpeps::g_prof_on = enable != 0;
  return FPEPS_OK;
}

fpeps_status fpeps_profile_read(int32_t kind, int64_t* launches, double* ms, double* flops, double* bytes) {
  if (kind < 0 || kind >= fpeps::PROF_KINDS || !launches || !ms || !flops || !bytes) return FPEPS_ERR_ARG;
  std::lock_guard<std::mutex> lk(fpeps::g_prof_mu);
  double t = 0, f = 0, b = 0;
  for (auto& r : fpeps::g_prof[kind]) {
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return FPEPS_ERR_CUDA;
    float x = 0;
    if (cudaEventElapsedTime(&x, r.e0, r.e1) != cudaSuccess) return FPEPS_ERR_CUDA;
    t += x;
    f += r.flops;
    b += r.bytes;
  }
  *launches = (int64_t)fpeps::g_prof[kind].size();
  *ms = t;
  *flops = f;
  *bytes = b;
  return FPEPS_OK;
}

const char* fpeps_version(void) { return "fpeps-gb300 0.1 (sm_103a)"; }

}  // extern "C"
