// The site sandwich C = A (x) W (x) A applied to blocks of vectors (Sec. III).
//
// The paper computes and stores the sandwich but advises against fusing the
// PEPO indices, because PEPO tensors of local Hamiltonians have structure
// beyond quantum-number conservation. Here the PEPO enters channel by channel:
// only the nonzero (l_w,u_w,r_w,d_w) blocks W_ch[p,p'] are visited, with the
// ket and the PEPO block pre-multiplied (A . W_ch), and the bra applied once
// per output (v_w, z_w) pair. C itself is never materialised.
//
// A block of the input, I[X][Y] with X = (x, x_w, x'), Y = (y, y_w, y')
// (bra fastest), maps to O[V][Z] with V = (v, v_w, v'), Z = (z, z_w, z'):
//   acc[x',y',v,z,q]   = sum_{ch in (v_w,z_w)} sum_{x,y} I[(x,x_w,x'),(y,y_w,y')] AW_ch[x,y,v,z,q]
//   O[(v,v_w,v'),(z,z_w,z')] = sum_{x',y',q} acc[x',y',v,z,q] A[x',y',v',z',q]
#include <algorithm>

#include "common.cuh"

namespace fpeps {
namespace {

template <class T>
__global__ void k_pepo_scan(const T* W, int n_ch, int pp, int* flags) {
  int ch = blockIdx.x * blockDim.x + threadIdx.x;
  if (ch >= n_ch) return;
  int f = 0;
  for (int i = 0; i < pp; ++i) f |= (W[(int64_t)ch * pp + i] != T(0));
  flags[ch] = f;
}

// index of a 4-leg site tensor element from role-ordered leg values
__device__ __forceinline__ int64_t leg_index(const int* dims, const int* roles, const int* vals) {
  int l[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) l[roles[r]] = vals[r];
  return (((int64_t)l[0] * dims[1] + l[1]) * dims[2] + l[2]) * dims[3] + l[3];
}

struct PrepArgs {
  int dA[5];
  int dW[6];
  int roles[4];
};

template <class T>
__global__ void k_prepare_ar(const T* A, PrepArgs a, T* ar) {
  const int nx = a.dA[a.roles[0]], ny = a.dA[a.roles[1]], nv = a.dA[a.roles[2]], nz = a.dA[a.roles[3]];
  const int p = a.dA[4];
  int64_t n = (int64_t)nx * ny * nv * nz * p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e;
    int q = r % p; r /= p;
    int z = r % nz; r /= nz;
    int v = r % nv; r /= nv;
    int y = r % ny; r /= ny;
    int x = (int)r;
    int vals[4] = {x, y, v, z};
    ar[e] = A[leg_index(a.dA, a.roles, vals) * p + q];
  }
}

template <class T>
__global__ void k_prepare_aw(const T* ar, const T* W, PrepArgs a, const int* ch, int nch, T* aw) {
  const int nx = a.dA[a.roles[0]], ny = a.dA[a.roles[1]], nv = a.dA[a.roles[2]], nz = a.dA[a.roles[3]];
  const int p = a.dA[4];
  const int64_t per = (int64_t)nx * ny * nv * nz * p;
  const int64_t n = per * nch;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(e / per);
    int64_t r = e % per;
    int q = r % p;
    int64_t base = r - q;   // element (x,y,v,z,0) of ar
    int wv[4] = {ch[4 * c + 0], ch[4 * c + 1], ch[4 * c + 2], ch[4 * c + 3]};
    int64_t wch = leg_index(a.dW, a.roles, wv) * p * p;   // W[l,u,r,d,:,:]
    T s = T(0);
    for (int pi = 0; pi < p; ++pi) s += ar[base + pi] * W[wch + (int64_t)pi * p + q];
    aw[e] = s;
  }
}

template <class T>
__global__ void k_first_row(const T* A, PrepArgs a, const T* W, T* out) {
  // T[L][Dn][R], L=(l,lw,l'), Dn=(d,dw,d'), R=(r,rw,r'); up legs have dimension 1
  const int Dl = a.dA[0], Dr = a.dA[2], Dd = a.dA[3], p = a.dA[4];
  const int wl = a.dW[0], wr = a.dW[2], wd = a.dW[3];
  const int64_t nL = (int64_t)Dl * wl * Dl, nD = (int64_t)Dd * wd * Dd, nR = (int64_t)Dr * wr * Dr;
  const int64_t n = nL * nD * nR;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t R = e % nR, Dn = (e / nR) % nD, L = e / (nR * nD);
    int rb = R % Dr, rw = (R / Dr) % wr, rk = R / (Dr * wr);
    int db = Dn % Dd, dw = (Dn / Dd) % wd, dk = Dn / (Dd * wd);
    int lb = L % Dl, lw = (L / Dl) % wl, lk = L / (Dl * wl);
    const T* ak = A + ((((int64_t)lk * 1 + 0) * Dr + rk) * Dd + dk) * p;
    const T* ab = A + ((((int64_t)lb * 1 + 0) * Dr + rb) * Dd + db) * p;
    const T* w = W + ((((int64_t)lw * 1 + 0) * wr + rw) * wd + dw) * p * p;
    T s = T(0);
    for (int i = 0; i < p; ++i) {
      T t = T(0);
      for (int j = 0; j < p; ++j) t += w[i * p + j] * ab[j];
      s += ak[i] * t;
    }
    out[e] = s;
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_sandwich(SandOrient o, int64_t nk, const T* __restrict__ in, int64_t i_t,
                                                  int64_t i_k, int64_t i_X, int64_t i_Y, T* __restrict__ out,
                                                  int64_t o_t, int64_t o_k, int64_t o_V, int64_t o_Z) {
  extern __shared__ unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int nx = o.nx, ny = o.ny, nv = o.nv, nz = o.nz, p = o.p;
  const int nsl = nx * nx * ny * ny;          // I slice [x][x'][y][y']
  const int nacc = nx * ny * nv * nz * p;     // acc [x'][y'][v][z][q] and ar/aw [x][y][v][z][q]
  T* isl = sm;
  T* acc = isl + nsl;
  T* ar = acc + nacc;
  T* aw = ar + nacc;
  const T* AW = static_cast<const T*>(o.d_aw);
  const T* AR = static_cast<const T*>(o.d_ar);

  const int64_t blk = blockIdx.x;
  const int64_t t = blk / nk, k = blk % nk;
  const T* I = in + t * i_t + k * i_k;
  T* O = out + t * o_t + k * o_k;
  const int tid = threadIdx.x;
  const bool pv = o_V == 1, pz = o_Z == 1 && o_V != 1;   // the unit-stride output bundle: PEPO outermost

  for (int e = tid; e < nacc; e += blockDim.x) ar[e] = AR[e];

  for (int vw = 0; vw < o.nvw; ++vw) {
    for (int zw = 0; zw < o.nzw; ++zw) {
      const int pair = vw * o.nzw + zw;
      const int c0 = o.d_pair_off[pair], c1 = o.d_pair_off[pair + 1];
      if (c0 == c1) {   // no PEPO channel feeds this output pair: zeros
        for (int e = tid; e < nv * nv * nz * nz; e += blockDim.x) {
          int zp = e % nz, z = (e / nz) % nz, vp = (e / (nz * nz)) % nv, v = e / (nz * nz * nv);
          const int64_t V = bundle_index(v, vw, vp, nv, o.nvw, pv);
          const int64_t Z = bundle_index(z, zw, zp, nz, o.nzw, pz);
          O[V * o_V + Z * o_Z] = T(0);
        }
        continue;
      }
      for (int e = tid; e < nacc; e += blockDim.x) acc[e] = T(0);
      for (int c = c0; c < c1; ++c) {
        const int xw = o.d_ch[4 * c + 0], yw = o.d_ch[4 * c + 1];
        __syncthreads();
        for (int e = tid; e < nsl; e += blockDim.x) {
          int yp = e % ny, y = (e / ny) % ny, xp = (e / (ny * ny)) % nx, x = e / (ny * ny * nx);
          int64_t X = ((int64_t)x * o.nxw + xw) * nx + xp;
          int64_t Y = ((int64_t)y * o.nyw + yw) * ny + yp;
          isl[e] = I[X * i_X + Y * i_Y];
        }
        const T* awc = AW + (int64_t)c * nacc;
        for (int e = tid; e < nacc; e += blockDim.x) aw[e] = awc[e];
        __syncthreads();
        // acc[x'][y'][v][z][q] += sum_{x,y} isl[x][x'][y][y'] aw[x][y][v][z][q]
        const int nvzq = nv * nz * p;
        for (int e = tid; e < nacc; e += blockDim.x) {
          int vzq = e % nvzq, yp = (e / nvzq) % ny, xp = e / (nvzq * ny);
          T s = T(0);
          for (int x = 0; x < nx; ++x)
            for (int y = 0; y < ny; ++y)
              s += isl[((x * nx + xp) * ny + y) * ny + yp] * aw[(x * ny + y) * nvzq + vzq];
          acc[e] += s;
        }
      }
      __syncthreads();
      // O[(v,vw,v'),(z,zw,z')] = sum_{x',y',q} acc[x'][y'][v][z][q] ar[x'][y'][v'][z'][q]
      const int nout = nv * nv * nz * nz;
      for (int e = tid; e < nout; e += blockDim.x) {
        int zp = e % nz, z = (e / nz) % nz, vp = (e / (nz * nz)) % nv, v = e / (nz * nz * nv);
        T s = T(0);
        for (int xp = 0; xp < nx; ++xp)
          for (int yp = 0; yp < ny; ++yp) {
            const T* ac = acc + ((xp * ny + yp) * nv + v) * nz * p + z * p;
            const T* br = ar + ((xp * ny + yp) * nv + vp) * nz * p + zp * p;
            for (int q = 0; q < p; ++q) s += ac[q] * br[q];
          }
        const int64_t V = bundle_index(v, vw, vp, nv, o.nvw, pv);
        const int64_t Z = bundle_index(z, zw, zp, nz, o.nzw, pz);
        O[V * o_V + Z * o_Z] = s;
      }
      __syncthreads();
    }
  }
}


// ---------------------------------------------------------------------------
// Tensor-core sandwich (3xTF32 with warp-level mma.sync m16n8k8): a CTA takes
// NB consecutive (t, k) blocks, so that the ket step is one small GEMM with
// rows (b, x', y') (<= 144 = 9 m16 tiles), K = (x, y) padded to a multiple of 8
// (<= 40) and N = (v, z, q) (<= 144 = 18 n8 tiles), accumulated over the
// channels of one output (v_w, z_w) pair; the accumulator is written to shared
// memory transposed to rows (b, v, z), K = (x', y', q) for the bra GEMM with
// N = (v', z') (<= 40). Every operand is split x = hi + lo (TF32 round to
// nearest) and the three products hi*hi + hi*lo + lo*hi accumulate in FP32.
constexpr int SM_MT = 9, SM_PA = 44, SM_PB = 152, SM_PC = 148, SM_PR = 40;
constexpr int SM_THREADS = 288;   // 9 warps
constexpr int SM_A = 144 * SM_PA, SM_B = 40 * SM_PB, SM_C = 144 * SM_PC, SM_R = 144 * SM_PR;
constexpr int SM_TILE_FLOATS = 2 * SM_A + 2 * SM_B + SM_C + SM_R;
constexpr int SM_FLOATS = SM_TILE_FLOATS + 2 * (144 + 144) + 144 + 2 * 144;   // + row tables, A / C offsets

// round to the nearest TF32 value, ties away from zero, with integer operations
// on the bit pattern (sign-magnitude: adding half an ulp to the magnitude)
__device__ __forceinline__ uint32_t to_tf32(float x) { return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u; }
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32_16x8x8(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// 3xTF32 products of split fragments: the three passes run over all tiles in
// turn, so consecutive MMAs never update the same accumulator
template <int MI, int NJ>
__device__ __forceinline__ void mma3_tiles(float (*acc)[NJ][4], const uint32_t (*ah)[4], const uint32_t (*al)[4],
                                           const uint32_t (*bh)[2], const uint32_t (*bl)[2]) {
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) mma_tf32_16x8x8(acc[i][j], al[i], bh[j]);
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) mma_tf32_16x8x8(acc[i][j], ah[i], bl[j]);
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) mma_tf32_16x8x8(acc[i][j], ah[i], bh[j]);
}

// The kernel is persistent (one CTA per SM walks the groups of nb_per blocks).
// Per group, offset tables give the input position of every (block, ket column
// (x, y)) and the output position of every (block, ket (v, z)); each thread keeps
// one bra position (x', y') for the gathers and one (v', z') for the stores, with
// the contiguous bundle index fastest across the lanes. The gathers of a channel
// are cp.async copies into one of two A/B buffers, issued while the MMAs of the
// previous channel run; the output tile is staged in shared memory.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(SM_THREADS, 1) k_sandwich_mma(SandOrient o, int64_t nt, int64_t nk, int nb_per,
                                                                int64_t ngroups, const float* __restrict__ in,
                                                                int64_t i_t, int64_t i_k, int64_t i_X, int64_t i_Y,
                                                                float* __restrict__ out, int64_t o_t, int64_t o_k,
                                                                int64_t o_V, int64_t o_Z) {
  extern __shared__ float sm[];
  float* const sA0 = sm;                    // A buffer b at sA0 + b * SM_A: rows (blk, x', y'), cols (x, y)
  float* const sB0 = sm + 2 * SM_A;         // B buffer b at sB0 + b * SM_B: rows (x, y), cols (v, z, q)
  float* const sC = sB0 + 2 * SM_B;         // rows (blk, v, z), cols (x', y', q)
  float* const sR = sC + SM_C;              // rows (x', y', q), cols (v', z')
  int64_t* const rowIn = reinterpret_cast<int64_t*>(sR + SM_R);   // [blk][x y] input offset
  int64_t* const rowOut = rowIn + 144;                            // [blk][v z] output offset
  int* const dstA = reinterpret_cast<int*>(rowOut + 144);         // [blk][x y] A-tile offset
  int* const cRow = dstA + 144;   // sC offset of ket accumulator row m = (blk, x', y')
  int* const cCol = cRow + 144;   // sC offset of ket accumulator column n = (v, z, q)
  const float* AW = static_cast<const float*>(o.d_aw);
  const float* AR = static_cast<const float*>(o.d_ar);
  const int nx = o.nx, ny = o.ny, nv = o.nv, nz = o.nz, p = o.p;
  const int K1 = nx * ny, N1 = nv * nz * p, K2 = nx * ny * p, N2 = nv * nz;
  const int K1p = (K1 + 7) & ~7, K2p = (K2 + 7) & ~7;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int g = lane >> 2, q4 = lane & 3;
  const int mg = warp / 3, ng = warp % 3;
  const int64_t nblk = nt * nk;
  const bool aw16 = (N1 % 4) == 0 && ((uintptr_t)AW % 16) == 0;
  // output strides of v, v_w (z, z_w): the unit-stride output bundle is PEPO-index outermost
  const bool pv = o_V == 1, pz = o_Z == 1 && o_V != 1;
  const int64_t sv = pv ? nv : (int64_t)o.nvw * nv, swv = pv ? (int64_t)nv * nv : nv;
  const int64_t sz = pz ? nz : (int64_t)o.nzw * nz, swz = pz ? (int64_t)nz * nz : nz;

  // this thread's gather slot: bra position (x', y'), lanes along the contiguous one
  const int gstep = SM_THREADS / K1, gslot = tid % K1, g0 = tid / K1;
  const bool gact = tid < gstep * K1;
  const bool x_fast = (i_X == 1 && i_Y != 1);
  const int gxp = x_fast ? gslot % nx : gslot / ny, gyp = x_fast ? gslot / nx : gslot % ny;
  const int64_t gpart = gxp * i_X + gyp * i_Y;
  const int grow = (gxp * ny + gyp) * SM_PA;
  // this thread's store slot: (v', z'), lanes along the contiguous one
  const int wstep = SM_THREADS / N2, wslot = tid % N2, w0 = tid / N2;
  const bool wact = tid < wstep * N2;
  const bool v_fast = (o_V == 1 && o_Z != 1);
  const int wvp = v_fast ? wslot % nv : wslot / nz, wzp = v_fast ? wslot / nv : wslot % nz;
  const int64_t wpart = wvp * o_V + wzp * o_Z;
  const int wcol = wvp * nz + wzp;

  for (int e = tid; e < SM_TILE_FLOATS; e += SM_THREADS) sm[e] = 0.f;
  __syncthreads();
  // sC[(blk N2 + vz) SM_PC + xy p + q] = cRow[m] + cCol[n] for m = (blk, xy), n = (vz, q)
  for (int e = tid; e < 144; e += SM_THREADS) {
    cRow[e] = (e / K1) * N2 * SM_PC + (e % K1) * p;
    cCol[e] = (e / p) * SM_PC + e % p;
  }
  for (int e = tid; e < K2 * N2; e += SM_THREADS) {
    int r = e / N2, c = e % N2;            // r = (x', y', q), c = (v', z')
    int q = r % p, xy = r / p, yp = xy % ny, xp = xy / ny;
    int zp = c % nz, vp = c / nz;
    sR[r * SM_PR + c] = AR[(((xp * ny + yp) * nv + vp) * nz + zp) * p + q];
  }

  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t b0 = grp * nb_per;
    const int nb = (int)min((int64_t)nb_per, nblk - b0);
    const int M1 = nb * K1, M2 = nb * N2;
    __syncthreads();   // the previous group is done with every table and tile
    for (int e = tid; e < M1; e += SM_THREADS) {
      const int bi = e / K1, col = e % K1, x = col / ny, y = col % ny;
      const int64_t b = b0 + bi, t = b / nk, k = b % nk;
      rowIn[e] = t * i_t + k * i_k + (int64_t)x * o.nxw * nx * i_X + (int64_t)y * o.nyw * ny * i_Y;
      dstA[e] = bi * K1 * SM_PA + col;
    }
    for (int e = tid; e < M2; e += SM_THREADS) {
      const int bi = e / N2, vz = e % N2, v = vz / nz, z = vz % nz;
      const int64_t b = b0 + bi, t = b / nk, k = b % nk;
      rowOut[e] = t * o_t + k * o_k + (int64_t)v * sv * o_V + (int64_t)z * sz * o_Z;
    }
    __syncthreads();

    // gathers of channel c into buffer buf (cp.async)
    auto issue = [&](int c, int buf) {
      const int xw = o.d_ch[4 * c + 0], yw = o.d_ch[4 * c + 1];
      if (gact) {
        const float* src = in + (int64_t)xw * nx * i_X + (int64_t)yw * ny * i_Y + gpart;
        float* A = sA0 + buf * SM_A + grow;
        for (int e = g0; e < M1; e += gstep) cp_async4(A + dstA[e], src + rowIn[e]);
      }
      const float* awc = AW + (int64_t)c * K1 * N1;
      float* Bm = sB0 + buf * SM_B;
      if (aw16) {
        const int n4 = N1 / 4;
        for (int e = tid; e < K1 * n4; e += SM_THREADS) {
          const int r = e / n4, c4 = e % n4;
          cp_async16(Bm + r * SM_PB + 4 * c4, awc + (int64_t)r * N1 + 4 * c4);
        }
      } else {
        for (int r = warp; r < K1; r += SM_THREADS / 32)
          for (int n = lane; n < N1; n += 32) cp_async4(Bm + r * SM_PB + n, awc + (int64_t)r * N1 + n);
      }
    };

    // output pairs with the contiguous bundle's channel index innermost, so that
    // consecutive pairs store adjacent bundle runs while they are still in L2
    const int nouter = v_fast ? o.nzw : o.nvw, ninner = v_fast ? o.nvw : o.nzw;
    for (int po = 0; po < nouter; ++po) {
      for (int pi = 0; pi < ninner; ++pi) {
        const int vw = v_fast ? pi : po, zw = v_fast ? po : pi;
        const int pair = vw * o.nzw + zw;
        const int c0 = o.d_pair_off[pair], c1 = o.d_pair_off[pair + 1];
        const int64_t obase = (int64_t)vw * swv * o_V + (int64_t)zw * swz * o_Z + wpart;
        if (c0 == c1) {   // no PEPO channel feeds this output pair: zeros
          if (wact)
            for (int e = w0; e < M2; e += wstep) out[rowOut[e] + obase] = 0.f;
          continue;
        }
        float acc[3][6][4];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 6; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
        __syncthreads();   // both A/B buffers free (previous pair's MMAs and output staging done)
        issue(c0, 0);
        cp_async_commit();
        for (int c = c0; c < c1; ++c) {
          const int buf = (c - c0) & 1;
          if (c + 1 < c1) {
            issue(c + 1, buf ^ 1);
            cp_async_commit();
            cp_async_wait<1>();
          } else {
            cp_async_wait<0>();
          }
          __syncthreads();
          const float* sA = sA0 + buf * SM_A;
          const float* sB = sB0 + buf * SM_B;
          for (int k0 = 0; k0 < K1p; k0 += 8) {
            uint32_t ah[3][4], al[3][4], bh[6][2], bl[6][2];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              const int r0 = (mg * 3 + i) * 16 + g;
              split_tf32(sA[r0 * SM_PA + k0 + q4], ah[i][0], al[i][0]);
              split_tf32(sA[(r0 + 8) * SM_PA + k0 + q4], ah[i][1], al[i][1]);
              split_tf32(sA[r0 * SM_PA + k0 + q4 + 4], ah[i][2], al[i][2]);
              split_tf32(sA[(r0 + 8) * SM_PA + k0 + q4 + 4], ah[i][3], al[i][3]);
            }
#pragma unroll
            for (int j = 0; j < 6; ++j) {
              const int n = (ng * 6 + j) * 8 + g;
              split_tf32(sB[(k0 + q4) * SM_PB + n], bh[j][0], bl[j][0]);
              split_tf32(sB[(k0 + q4 + 4) * SM_PB + n], bh[j][1], bl[j][1]);
            }
            mma3_tiles<3, 6>(acc, ah, al, bh, bl);
          }
          __syncthreads();   // this buffer is refilled two channels later
        }
        // acc (rows (bi,x',y'), cols (v,z,q)) -> sC rows (bi,v,z), cols (x',y',q)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 6; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int m = (mg * 3 + i) * 16 + g + ((r >> 1) << 3);
              const int n = (ng * 6 + j) * 8 + q4 * 2 + (r & 1);
              if (m < M1 && n < N1) sC[cRow[m] + cCol[n]] = acc[i][j][r];
            }
        __syncthreads();
        // bra: rows (bi, v, z) x cols (v', z'), K = (x', y', q)
        // two accumulator sets over alternating k-steps: 10 independent MMA chains
        float d2[2][5][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int j = 0; j < 5; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) d2[u][j][r] = 0.f;
        const int r0 = warp * 16 + g;
        auto bra_step = [&](int kk, uint32_t(&ah)[1][4], uint32_t(&al)[1][4], uint32_t(&bh)[5][2],
                            uint32_t(&bl)[5][2]) {
          split_tf32(sC[r0 * SM_PC + kk + q4], ah[0][0], al[0][0]);
          split_tf32(sC[(r0 + 8) * SM_PC + kk + q4], ah[0][1], al[0][1]);
          split_tf32(sC[r0 * SM_PC + kk + q4 + 4], ah[0][2], al[0][2]);
          split_tf32(sC[(r0 + 8) * SM_PC + kk + q4 + 4], ah[0][3], al[0][3]);
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            split_tf32(sR[(kk + q4) * SM_PR + j * 8 + g], bh[j][0], bl[j][0]);
            split_tf32(sR[(kk + q4 + 4) * SM_PR + j * 8 + g], bh[j][1], bl[j][1]);
          }
        };
        int k0 = 0;
        for (; k0 + 16 <= K2p; k0 += 16) {
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            uint32_t ah0[1][4], al0[1][4], bh0[5][2], bl0[5][2];
            bra_step(k0 + 8 * u, ah0, al0, bh0, bl0);
            mma3_tiles<1, 5>(&d2[u], ah0, al0, bh0, bl0);
          }
        }
        if (k0 < K2p) {   // K2p / 8 odd: one k-step left
          uint32_t ah0[1][4], al0[1][4], bh0[5][2], bl0[5][2];
          bra_step(k0, ah0, al0, bh0, bl0);
          mma3_tiles<1, 5>(&d2[0], ah0, al0, bh0, bl0);
        }
        // stage the output tile in A buffer 0 (free): rows (bi, v, z), cols (v', z')
        float* st = sA0;
#pragma unroll
        for (int j = 0; j < 5; ++j)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int m = warp * 16 + g + ((r >> 1) << 3);
            const int n = j * 8 + q4 * 2 + (r & 1);
            if (m < M2 && n < N2) st[m * SM_PA + n] = d2[0][j][r] + d2[1][j][r];
          }
        __syncthreads();
        if (wact)
          for (int e = w0; e < M2; e += wstep) out[rowOut[e] + obase] = st[e * SM_PA + wcol];
      }
    }
  }
}

int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 152 * 64 ? 152 * 64 : (g < 1 ? 1 : g));
}

}  // namespace

template <class T>
void pepo_scan(cudaStream_t s, const T* W, const int dW[6], int* d_flags) {
  int nch = dW[0] * dW[1] * dW[2] * dW[3];
  k_pepo_scan<T><<<(nch + 127) / 128, 128, 0, s>>>(W, nch, dW[4] * dW[5], d_flags);
  FP_LAUNCH();
}

template <class T>
void sandwich_prepare(cudaStream_t s, const T* A, const int dA[5], const T* W, const int dW[6], const int roles[4],
                      const int* d_ch, int nch, T* d_aw, T* d_ar) {
  PrepArgs a;
  for (int i = 0; i < 5; ++i) a.dA[i] = dA[i];
  for (int i = 0; i < 6; ++i) a.dW[i] = dW[i];
  for (int i = 0; i < 4; ++i) a.roles[i] = roles[i];
  int64_t per = (int64_t)dA[roles[0]] * dA[roles[1]] * dA[roles[2]] * dA[roles[3]] * dA[4];
  k_prepare_ar<T><<<grid_for(per), 256, 0, s>>>(A, a, d_ar);
  FP_LAUNCH();
  if (nch > 0) {
    k_prepare_aw<T><<<grid_for(per * nch), 256, 0, s>>>(d_ar, W, a, d_ch, nch, d_aw);
    FP_LAUNCH();
  }
}

template <class T>
void first_row_tensor(cudaStream_t s, const T* A, const int dA[5], const T* W, const int dW[6], T* out) {
  PrepArgs a;
  for (int i = 0; i < 5; ++i) a.dA[i] = dA[i];
  for (int i = 0; i < 6; ++i) a.dW[i] = dW[i];
  int64_t n = (int64_t)dA[0] * dW[0] * dA[0] * dA[3] * dW[3] * dA[3] * dA[2] * dW[2] * dA[2];
  k_first_row<T><<<grid_for(n), 256, 0, s>>>(A, a, W, out);
  FP_LAUNCH();
}

bool sandwich_mma_fits(const SandOrient& o) {
  const int K1 = o.nx * o.ny, N1 = o.nv * o.nz * o.p, K2 = K1 * o.p, N2 = o.nv * o.nz;
  return K1 <= 40 && N1 <= 144 && K2 <= 144 && N2 <= 40 && K1 >= 1 && N2 >= 1 && o.nx <= 6 && o.ny <= 6 &&
         o.nv <= 6 && o.nz <= 6;   // offset tables hold 36 entries
}

void sandwich_apply_tc(cudaStream_t s, const SandOrient& o, int64_t nt, int64_t nk, const float* in, int64_t i_t,
                       int64_t i_k, int64_t i_X, int64_t i_Y, float* out, int64_t o_t, int64_t o_k, int64_t o_V,
                       int64_t o_Z) {
  if (nt <= 0 || nk <= 0) return;
  FP_CHECK(sandwich_mma_fits(o), FPEPS_ERR_UNSUPPORTED, "tensor-core sandwich: site dimensions too large");
  const int K1 = o.nx * o.ny, N2 = o.nv * o.nz;
  const int nb_per = std::max(1, std::min(144 / K1, 144 / N2));
  const int64_t nblk = nt * nk;
  const int64_t ngroups = (nblk + nb_per - 1) / nb_per;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    FP_CUDA(cudaGetDevice(&dev));
    FP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t grid = std::min<int64_t>(ngroups, sms);
  const size_t smem = (size_t)SM_FLOATS * sizeof(float);
  static bool attr = false;
  if (!attr) {
    FP_CUDA(cudaFuncSetAttribute(k_sandwich_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_sandwich_mma<<<(unsigned)grid, SM_THREADS, smem, s>>>(o, nt, nk, nb_per, ngroups, in, i_t, i_k, i_X, i_Y, out,
                                                          o_t, o_k, o_V, o_Z);
  FP_LAUNCH();
}

template <class T>
void sandwich_apply(cudaStream_t s, const SandOrient& o, int64_t nt, int64_t nk, const T* in, int64_t i_t,
                    int64_t i_k, int64_t i_X, int64_t i_Y, T* out, int64_t o_t, int64_t o_k, int64_t o_V,
                    int64_t o_Z) {
  if (nt <= 0 || nk <= 0) return;
  size_t nsl = (size_t)o.nx * o.nx * o.ny * o.ny;
  size_t nacc = (size_t)o.nx * o.ny * o.nv * o.nz * o.p;
  size_t smem = (nsl + 3 * nacc) * sizeof(T);
  FP_CHECK(smem <= 200 * 1024, FPEPS_ERR_UNSUPPORTED, "sandwich: site too large for shared memory");
  static bool attr_set[2] = {false, false};
  int idx = sizeof(T) == 8 ? 1 : 0;
  if (!attr_set[idx]) {
    FP_CUDA(cudaFuncSetAttribute(k_sandwich<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[idx] = true;
  }
  int64_t nblk = nt * nk;
  FP_CHECK(nblk < (1LL << 31), FPEPS_ERR_UNSUPPORTED, "sandwich: too many blocks");
  k_sandwich<T><<<(unsigned)nblk, 256, smem, s>>>(o, nk, in, i_t, i_k, i_X, i_Y, out, o_t, o_k, o_V, o_Z);
  FP_LAUNCH();
}

#define INST(T)                                                                                                   \
  template void pepo_scan<T>(cudaStream_t, const T*, const int[6], int*);                                        \
  template void sandwich_prepare<T>(cudaStream_t, const T*, const int[5], const T*, const int[6], const int[4],  \
                                    const int*, int, T*, T*);                                                     \
  template void first_row_tensor<T>(cudaStream_t, const T*, const int[5], const T*, const int[6], T*);          \
  template void sandwich_apply<T>(cudaStream_t, const SandOrient&, int64_t, int64_t, const T*, int64_t, int64_t, \
                                  int64_t, int64_t, T*, int64_t, int64_t, int64_t, int64_t);
INST(float)
INST(double)

}  // namespace fpeps
