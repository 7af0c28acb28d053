// Environment state shared by the runtime (abi.cu) and the row engine (engine.cu).
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "common.cuh"

namespace fpeps {

enum class RowState { Ready, Staged, Closed };

// Device copy of one lattice site (compute precision) and its sandwich data.
struct SiteHost {
  int dA[5];   // Dl, Du, Dr, Dd, p
  int dW[6];   // wl, wu, wr, wd, p, p'
  size_t offA = 0, offW = 0;   // element offsets into the packed device buffers
  // channels of the PEPO site in (l,u,r,d) order
  std::vector<int> ch;   // 4 ints per channel
  // block-sparse mode: U(1) x U(1) charges (N_up, N_dn) of the (ket, PEPO, bra)
  // bundles of legs l, u, r, d, bra fastest: Q = q_ket - q_pepo - q_bra
  std::vector<int32_t> qB[4];
};

// Sandwich data of one site for the four orientations (device memory, per layer).
struct SiteSand {
  SandOrient o[4];
  std::vector<void*> bufs;   // owned device buffers
  int n_ld = 0;              // nonzero (v_w, z_w) pairs in FWD orientation
};

struct Spectrum {
  std::vector<std::vector<double>> zip, fit;
};

struct EngineBase;

}  // namespace fpeps

struct fpeps_env {
  fpeps_config cfg{};
  int elem = 8;                  // bytes per element of the compute precision
  cudaStream_t stream = nullptr;
  fpeps::Allocator al;
  bool poisoned = false;
  std::string err;

  // packed site tensors (device, compute precision)
  void* peps = nullptr;
  void* pepo[2] = {nullptr, nullptr};   // [0] identity, [1] operator (may be null)
  std::vector<fpeps::SiteHost> sites[2];   // per layer, Lx*Ly
  std::vector<fpeps::SiteSand> sand[2];    // per layer, Lx*Ly (built lazily)

  // boundary MPS: T_c [t_{c-1}][U_c][t_c]
  std::vector<void*> T;
  std::vector<int> tb;      // Ly+1 bond dims
  std::vector<int> tphys;   // Ly phys (bundle) dims
  std::vector<std::vector<int32_t>> qT;   // block-sparse mode: charges of the Ly+1 bonds (pairs)
  double log_scale = 0.0;   // ln of the scale taken out of the boundary so far
  int next_row = 0;
  int layer = 0;
  fpeps::RowState state = fpeps::RowState::Ready;
  int staged_row = -1;
  bool have_value = false;
  double value_log = 0.0;
  int value_sign = 0;

  fpeps::Spectrum spectra;

  // n_envs > 1: independent environments over the same lattice. Each keeps its own
  // boundary, sweep state, value and spectra (the fields above, for the selected one;
  // the others parked here) and its own sketch streams (its index enters the generator
  // counter); the lattice, the staged sandwich data, the engine's scratch and the
  // stream are shared.
  struct Slot {
    std::vector<void*> T;
    std::vector<int> tb, tphys;
    std::vector<std::vector<int32_t>> qT;
    double log_scale = 0.0;
    int next_row = 0, layer = 0;
    fpeps::RowState state = fpeps::RowState::Ready;
    int staged_row = -1;
    bool have_value = false;
    double value_log = 0.0;
    int value_sign = 0;
    fpeps::Spectrum spectra;
  };
  std::vector<Slot> slots;   // n_envs entries; slots[cur] is stale while cur is selected
  int cur = 0;

  fpeps::EngineBase* engine = nullptr;
  int* d_info = nullptr;    // device status words
  int* h_info = nullptr;    // pinned host mirror
  double* d_scal = nullptr; // device scalars
  double* h_scal = nullptr;
};

namespace fpeps {

struct EngineBase {
  virtual ~EngineBase() {}
  virtual void first_row(fpeps_env* env, int row) = 0;
  virtual void close_row(fpeps_env* env, int row) = 0;
  virtual void compress(fpeps_env* env, int row, const fpeps_rsvd_params& prm, fpeps_stats* st) = 0;
  virtual void apply_theta_host(fpeps_env* env, int op, int c, int a, const void* envh, int k, const void* in,
                                void* out) = 0;
};

EngineBase* make_engine(fpeps_env* env);
void ensure_sandwich(fpeps_env* env, int layer, int row);

}  // namespace fpeps
