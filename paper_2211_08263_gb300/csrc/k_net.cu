// Learned warm start (not part of the paper's method; the paper's solver
// starts each step from u_{n-1}): network kernels, the GPU training loop and
// their C ABI entry points (include/wfft.h, "learned warm start").
//
// Network: 4 periodic 3x3x3 convolutions 16 -> H -> H -> H -> 3 (H = 16 or 32),
// ReLU after the first three.  Activations are channels-last [V][C] BF16, weights
// BF16, accumulation FP32 on the tensor cores (mma.sync m16n8k16 bf16), biases
// and the master parameters FP32.
//
// Convolution kernels are implicit GEMMs over (voxel tile) x (27 offsets x
// input channels): a CTA owns a 16 x 8 x 2 output tile, stages its periodic
// 18 x 10 x 4 input halo in shared memory with cp.async (rows swizzled so that
// ldmatrix reads are bank-conflict free) and keeps the layer's weights resident
// in shared memory across the tiles it visits (persistent grid).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "../../include/wfft.h"
#include "common.cuh"
#include "net.cuh"
#include "profiler.cuh"

namespace wfft {
void set_global_error(const char* msg);
}  // namespace wfft

using namespace wfft;

namespace {

typedef __nv_bfloat16 bf16;

// Set by a tcgen05 convolution whose bounded wait on the tensor cores expired.
__device__ int g_conv_tc_err;

constexpr int TX = 16, TY = 8, TZ = 2;            // output tile
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int HV = HX * HY * HZ;                   // halo voxels
constexpr int TV = TX * TY * TZ;                   // tile voxels
constexpr int kThreads = 256;

enum { EPI_RELU = 0, EPI_LINEAR, EPI_GRAD, EPI_WARM };

struct ConvArgs {
  int n1, n2, n3;
  long long V;
  int ntx, nty, ntz;
  long long ntiles;
  const bf16* in;      // [V][CIN]
  const bf16* W;       // [27][COUT][CIN]
  const float* bias;   // [COUT] (EPI_RELU / EPI_LINEAR / EPI_WARM)
  void* out;
  const bf16* gate;    // EPI_GRAD: forward activation [V][COUT]; wgrad: output gradient [V][COUT]
  // EPI_WARM
  int c;
  const double* v;
  const double* a;
  const uint8_t* mask;
  double dt;
  const float* scale;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
// D = A B + D, A 16x16 (row), B 16x8 (col), BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// 16-byte chunk j of row `row` of a [rows][C] BF16 tile is stored at chunk
// swz(row, j): any 8 consecutive rows then hit 8 distinct bank groups.
template <int C>
__device__ __forceinline__ int swz(int row, int j) {
  static_assert(C == 16 || C == 32, "channel count");
  return C == 16 ? (j ^ ((row >> 2) & 1)) : (j ^ ((row >> 1) & 3));
}

__device__ __forceinline__ int wrapi(int g, int n) {
  int r = g % n;
  return r < 0 ? r + n : r;
}

// Periodic coordinates of the halo of tile t: xs[HX], ys[HY], zs[HZ].
__device__ __forceinline__ void tile_origin(const ConvArgs& p, long long t, int& x0, int& y0, int& z0) {
  const int tx = (int)(t % p.ntx);
  const long long r = t / p.ntx;
  x0 = tx * TX;
  y0 = (int)(r % p.nty) * TY;
  z0 = (int)(r / p.nty) * TZ;
}
__device__ __forceinline__ void halo_tables(const ConvArgs& p, int x0, int y0, int z0, int* tab) {
  const int i = threadIdx.x;
  if (i < HX)
    tab[i] = wrapi(x0 - 1 + i, p.n1);
  else if (i < HX + HY)
    tab[i] = wrapi(y0 - 1 + (i - HX), p.n2);
  else if (i < HX + HY + HZ)
    tab[i] = wrapi(z0 - 1 + (i - HX - HY), p.n3);
}
template <int CIN>
__device__ __forceinline__ void load_halo(const ConvArgs& p, bf16* Hs, const int* tab) {
  constexpr int CH = CIN / 8;
  for (int id = threadIdx.x; id < HV * CH; id += blockDim.x) {
    const int hv = id / CH, j = id - hv * CH;
    const int hx = hv % HX, hy = (hv / HX) % HY, hz = hv / (HX * HY);
    const long long g = ((long long)tab[HX + HY + hz] * p.n2 + tab[HX + hy]) * p.n1 + tab[hx];
    cp16(smem_u32(Hs + hv * CIN + 8 * swz<CIN>(hv, j)), p.in + g * CIN + 8 * j);
  }
  cp_commit();
}

template <int CIN, int COUT>
constexpr size_t conv_smem() {
  return (size_t)27 * COUT * CIN * 2 + (size_t)HV * CIN * 2 + 32 * sizeof(int);
}

// out = epilogue(conv(in, W)) -- forward layers, the input-gradient of the
// backward pass (EPI_GRAD: W in the transposed / reversed layout, times the
// ReLU gate) and the warm start (EPI_WARM: dt v + dt^2/2 a + s (y + b) on
// free DOFs, written as an FP32 [c][V] field).
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kThreads, 2) k_conv(ConvArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  bf16* Ws = reinterpret_cast<bf16*>(sm);
  bf16* Hs = Ws + 27 * COUT * CIN;
  int* tab = reinterpret_cast<int*>(Hs + HV * CIN);
  constexpr int WCH = CIN / 8;
  for (int id = threadIdx.x; id < 27 * COUT * WCH; id += blockDim.x) {
    const int r = id / WCH, j = id - r * WCH;
    cp16(smem_u32(Ws + r * CIN + 8 * swz<CIN>(r, j)), p.W + (size_t)r * CIN + 8 * j);
  }
  cp_commit();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wz = warp >> 2, wy0 = (warp & 3) * 2;
  const int g = lane >> 2, q = (lane & 3) * 2;
  for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
    int x0, y0, z0;
    tile_origin(p, t, x0, y0, z0);
    halo_tables(p, x0, y0, z0, tab);
    __syncthreads();
    load_halo<CIN>(p, Hs, tab);
    cp_wait_all();
    __syncthreads();
    float acc[2][COUT / 8][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int n = 0; n < COUT / 8; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;
#pragma unroll 1
    for (int dz = 0; dz < 3; ++dz) {
      // the nine (y, x) offsets of a z offset unrolled: the next offset's fragment loads
      // can be issued under the current offset's MMAs
#pragma unroll
      for (int o9 = 0; o9 < 9; ++o9) {
      const int dy = o9 / 3, dx = o9 % 3;
      const int o = 9 * dz + o9;
#pragma unroll
      for (int ks = 0; ks < CIN / 16; ++ks) {
        uint32_t A[2][4];
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          const int hv = ((wz + dz) * HY + (wy0 + m + dy)) * HX + dx + (lane & 15);
          const int ch = 2 * ks + (lane >> 4);
          ldsm_x4(smem_u32(Hs + hv * CIN + 8 * swz<CIN>(hv, ch)), A[m]);
        }
#pragma unroll
        for (int np = 0; np < COUT / 16; ++np) {
          const int r = o * COUT + np * 16 + (lane & 7) + ((lane >> 4) << 3);
          const int ch = 2 * ks + ((lane >> 3) & 1);
          uint32_t B[4];
          ldsm_x4(smem_u32(Ws + r * CIN + 8 * swz<CIN>(r, ch)), B);
#pragma unroll
          for (int m = 0; m < 2; ++m) {
            mma_bf16(acc[m][2 * np], A[m], B[0], B[1]);
            mma_bf16(acc[m][2 * np + 1], A[m], B[2], B[3]);
          }
        }
      }
      }
    }
    // epilogue: accumulator (m, n, e) is voxel x0 + g + 8 (e >> 1) of row (wz, wy0 + m),
    // channel 8 n + q + (e & 1)
    const int z = z0 + wz;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int y = y0 + wy0 + m;
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int x = x0 + g + 8 * hf;
        if (x >= p.n1 || y >= p.n2 || z >= p.n3) continue;
        const long long vox = ((long long)z * p.n2 + y) * p.n1 + x;
#pragma unroll
        for (int n = 0; n < COUT / 8; ++n) {
          const int col = 8 * n + q;
          const float c0 = acc[m][n][2 * hf], c1 = acc[m][n][2 * hf + 1];
          if (EPI == EPI_RELU) {
            const float v0 = fmaxf(c0 + p.bias[col], 0.f), v1 = fmaxf(c1 + p.bias[col + 1], 0.f);
            reinterpret_cast<__nv_bfloat162*>(p.out)[(vox * COUT + col) >> 1] = __floats2bfloat162_rn(v0, v1);
          } else if (EPI == EPI_LINEAR) {
            if (col < 4)
              reinterpret_cast<float2*>(p.out)[(vox * 4 + col) >> 1] =
                  make_float2(c0 + p.bias[col], c1 + p.bias[col + 1]);
          } else if (EPI == EPI_GRAD) {
            const __nv_bfloat162 gt = reinterpret_cast<const __nv_bfloat162*>(p.gate)[(vox * COUT + col) >> 1];
            const float v0 = __low2float(gt) > 0.f ? c0 : 0.f, v1 = __high2float(gt) > 0.f ? c1 : 0.f;
            reinterpret_cast<__nv_bfloat162*>(p.out)[(vox * COUT + col) >> 1] = __floats2bfloat162_rn(v0, v1);
          } else {  // EPI_WARM: delta (the Taylor increment, 0 on Gamma) += s (y + b) on free DOFs
            if (col < p.c) {
              const float s = p.scale[0];
              const uint8_t mk = p.mask ? p.mask[vox] : (uint8_t)0;
              float* delta = reinterpret_cast<float*>(p.out);
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int k = col + e;
                if (k >= p.c || ((mk >> k) & 1)) continue;
                const long long gi = (long long)k * p.V + vox;
                delta[gi] = delta[gi] + s * ((e ? c1 : c0) + p.bias[k]);
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
  return (size_t)HV * CIN * 2 + (size_t)TV * COUT * 2 + 32 * sizeof(int);
}

// Weight and bias gradients of one layer: dW[o][co][ci] += sum_x G[x][co] in[x + off_o][ci],
// db[co] += sum_x G[x][co].  Voxels are the MMA reduction dimension (both operands
// through ldmatrix.trans); each warp owns offsets warp, warp + 8, ...; every tile
// adds its partial sums to dW with FP32 atomics.
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) k_conv_wgrad(ConvArgs p, float* dW, float* db) {
  extern __shared__ __align__(128) unsigned char sm[];
  bf16* Hs = reinterpret_cast<bf16*>(sm);
  bf16* Gs = Hs + HV * CIN;
  int* tab = reinterpret_cast<int*>(Gs + TV * COUT);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = (lane & 3) * 2;
  for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
    int x0, y0, z0;
    tile_origin(p, t, x0, y0, z0);
    halo_tables(p, x0, y0, z0, tab);
    __syncthreads();
    load_halo<CIN>(p, Hs, tab);
    constexpr int GCH = COUT / 8;
    for (int id = threadIdx.x; id < TV * GCH; id += blockDim.x) {
      const int lv = id / GCH, j = id - lv * GCH;
      const int x = x0 + (lv & 15), y = y0 + ((lv >> 4) & 7), z = z0 + (lv >> 7);
      bf16* dst = Gs + lv * COUT + 8 * swz<COUT>(lv, j);
      if (x < p.n1 && y < p.n2 && z < p.n3) {
        const long long vox = ((long long)z * p.n2 + y) * p.n1 + x;
        cp16(smem_u32(dst), p.gate + vox * COUT + 8 * j);
      } else {
        *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
      }
    }
    cp_commit();
    cp_wait_all();
    __syncthreads();
    if (threadIdx.x < COUT) {
      const int col = threadIdx.x, j = col >> 3, e = col & 7;
      float s = 0.f;
      for (int lv = 0; lv < TV; ++lv) s += __bfloat162float(Gs[lv * COUT + 8 * swz<COUT>(lv, j) + e]);
      atomicAdd(db + col, s);
    }
    for (int o = warp; o < 27; o += kThreads / 32) {
      const int dz = o / 9, dy = (o / 3) % 3, dx = o % 3;
      float acc[COUT / 16][CIN / 8][4];
#pragma unroll
      for (int a = 0; a < COUT / 16; ++a)
#pragma unroll
        for (int b = 0; b < CIN / 8; ++b)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.f;
#pragma unroll 2
      for (int r = 0; r < TY * TZ; ++r) {
        uint32_t A[COUT / 16][4];
#pragma unroll
        for (int mt = 0; mt < COUT / 16; ++mt) {
          const int lv = r * 16 + (lane & 7) + ((lane >> 4) << 3);
          const int ch = 2 * mt + ((lane >> 3) & 1);
          ldsm_x4_t(smem_u32(Gs + lv * COUT + 8 * swz<COUT>(lv, ch)), A[mt]);
        }
#pragma unroll
        for (int np = 0; np < CIN / 16; ++np) {
          const int hv = (((r >> 3) + dz) * HY + ((r & 7) + dy)) * HX + (lane & 15) + dx;
          const int ch = 2 * np + (lane >> 4);
          uint32_t B[4];
          ldsm_x4_t(smem_u32(Hs + hv * CIN + 8 * swz<CIN>(hv, ch)), B);
#pragma unroll
          for (int mt = 0; mt < COUT / 16; ++mt) {
            mma_bf16(acc[mt][2 * np], A[mt], B[0], B[1]);
            mma_bf16(acc[mt][2 * np + 1], A[mt], B[2], B[3]);
          }
        }
      }
#pragma unroll
      for (int mt = 0; mt < COUT / 16; ++mt)
#pragma unroll
        for (int nt = 0; nt < CIN / 8; ++nt) {
          float* w = dW + ((size_t)o * COUT + 16 * mt + g) * CIN + 8 * nt + q;
          atomicAdd(w, acc[mt][nt][0]);
          atomicAdd(w + 1, acc[mt][nt][1]);
          atomicAdd(w + 8 * CIN, acc[mt][nt][2]);
          atomicAdd(w + 8 * CIN + 1, acc[mt][nt][3]);
        }
    }
    __syncthreads();
  }
}

#include "conv_tc.cuh"

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------
constexpr int kAuxBlocks = 1216;

// Partial sums of the warm-start scale: sum (dt v)^2 + (dt^2/2 a)^2 over all DOFs
// plus (U_n - u - dt v - dt^2/2 a)^2 over the prescribed DOFs.
__global__ void __launch_bounds__(256) k_warm_scale(WarmArgs w, double* part) {
  double acc = 0.0;
  const double dt = w.dt, h2 = 0.5 * w.dt * w.dt;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < w.V;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t mk = w.mask ? w.mask[i] : (uint8_t)0;
    for (int k = 0; k < w.c; ++k) {
      const long long gi = (long long)k * w.V + i;
      const double dv = dt * w.v[gi], da = h2 * w.a[gi];
      acc += dv * dv + da * da;
      if ((mk >> k) & 1) {
        const double e = w.Ug[k] - (w.u[gi] + dv + da);
        acc += e * e;
      }
    }
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// s = sqrt(sum / (c V)); scale = {s, 1/s} (both 0 for a state at rest).
__global__ void k_warm_scale_fin(const double* part, int n, double cV, float* scale) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) {
    const double r = sqrt(s / cV);
    const bool ok = r > 1e-300 && isfinite(r);
    scale[0] = ok ? (float)r : 0.f;
    scale[1] = ok ? (float)(1.0 / r) : 0.f;
  }
}

// Input features (16 BF16 channels per voxel): dt v / s (3), dt^2/2 a / s (3),
// prescribed increment U_n - Taylor on Gamma / s (3), Gamma indicator, rho/rho_bar - 1,
// normal stiffnesses C_kk / C_bar_kk - 1 (3), shear and off-diagonal normal sums
// relative to their means - 1.
// Taylor part of the warm-start increment, dt v + dt^2/2 a, rounded once to FP32 (the
// same operations in every kernel that forms it, so the learned and Taylor warm starts
// agree bit for bit when the network's output is zero).
__device__ __forceinline__ float taylor_increment(double dt, double v, double a) {
  return (float)__fma_rn(dt, v, __dmul_rn(__dmul_rn(0.5 * dt, dt), a));
}

// Network input features and, into delta (when given), the Taylor increment on free DOFs
// (0 on Gamma), to which the last layer's epilogue adds the scaled network output.
__global__ void __launch_bounds__(256) k_warm_features(WarmArgs w, const float* scale, bf16* X, float* delta) {
  const float inv = scale[1];
  const double dt = w.dt, h2 = 0.5 * w.dt * w.dt;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < w.V;
       i += (long long)gridDim.x * blockDim.x) {
    float f[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) f[k] = 0.f;
    const uint8_t mk = w.mask ? w.mask[i] : (uint8_t)0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k >= w.c) continue;
      const long long gi = (long long)k * w.V + i;
      const double dv = dt * w.v[gi], da = h2 * w.a[gi];
      f[k] = (float)dv * inv;
      f[3 + k] = (float)da * inv;
      if ((mk >> k) & 1) f[6 + k] = (float)(w.Ug[k] - (w.u[gi] + dv + da)) * inv;
      if (delta) delta[gi] = ((mk >> k) & 1) ? 0.f : taylor_increment(dt, w.v[gi], w.a[gi]);
    }
    f[9] = mk ? 1.f : 0.f;
    const long long row = w.phase ? (long long)w.phase[i] : i;
    f[10] = w.rhotab[row] * w.inv_rhobar - 1.f;
    const float* C = w.ctab + row * w.cstride;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (w.nd_idx[k] >= 0) f[11 + k] = C[w.nd_idx[k]] * w.inv_nd[k] - 1.f;
    float sh = 0.f, of = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (w.sh_idx[k] >= 0) sh += C[w.sh_idx[k]];
      if (w.of_idx[k] >= 0) of += C[w.of_idx[k]];
    }
    f[14] = sh * w.inv_sh - 1.f;
    f[15] = w.inv_of != 0.f ? of * w.inv_of - 1.f : 0.f;
    uint32_t pk[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      __nv_bfloat162 b = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
      pk[k] = *reinterpret_cast<uint32_t*>(&b);
    }
    uint4* dst = reinterpret_cast<uint4*>(X + i * 16);
    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  }
}

// Taylor increment alone: delta = dt v + dt^2/2 a on free DOFs, 0 on Gamma.
__global__ void __launch_bounds__(256) k_warm_taylor(WarmArgs w, float* delta) {
  const long long tot = (long long)w.c * w.V;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < tot;
       gi += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(gi / w.V);
    const long long i = gi - (long long)k * w.V;
    const uint8_t mk = w.mask ? w.mask[i] : (uint8_t)0;
    delta[gi] = ((mk >> k) & 1) ? 0.f : taylor_increment(w.dt, w.v[gi], w.a[gi]);
  }
}

// Training target: (u_n - Taylor) / s = theta (a_n - a_{n-1}) / s on free DOFs, [V][4] FP32.
__global__ void __launch_bounds__(256) k_net_target(long long V, int c, const double* a_new, const double* a_old,
                                                    const uint8_t* mask, double theta, const float* scale,
                                                    float* T) {
  const double inv = scale[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    const uint8_t mk = mask ? mask[i] : (uint8_t)0;
    for (int k = 0; k < c; ++k)
      if (!((mk >> k) & 1)) t[k] = (float)(theta * (a_new[(long long)k * V + i] - a_old[(long long)k * V + i]) * inv);
    reinterpret_cast<float4*>(T)[i] = make_float4(t[0], t[1], t[2], t[3]);
  }
}

// Loss sum_free (y - t)^2 (added to *loss) and its gradient gs (y - t) as BF16 [V][16].
__global__ void __launch_bounds__(256) k_loss_grad(long long V, int c, const float* Y, const float* T,
                                                   const uint8_t* mask, float gs, bf16* G, double* loss) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    float gr[4] = {0.f, 0.f, 0.f, 0.f};
    const uint8_t mk = mask ? mask[i] : (uint8_t)0;
    for (int k = 0; k < c; ++k) {
      if ((mk >> k) & 1) continue;
      const float d = Y[i * 4 + k] - T[i * 4 + k];
      acc += (double)d * d;
      gr[k] = gs * d;
    }
    __nv_bfloat162 b0 = __floats2bfloat162_rn(gr[0], gr[1]), b1 = __floats2bfloat162_rn(gr[2], gr[3]);
    uint4* dst = reinterpret_cast<uint4*>(G + i * 16);
    dst[0] = make_uint4(*reinterpret_cast<uint32_t*>(&b0), *reinterpret_cast<uint32_t*>(&b1), 0u, 0u);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(loss, s);
}

__global__ void k_f32_to_bf16(const float* in, bf16* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// BF16 copies of the weights: forward layout W[o][co][ci] and, for training, the
// input-gradient layout Wt[26 - o][ci][co].
struct DimsDev {
  int cin[kNetLayers], cout[kNetLayers];
  long long woff[kNetLayers], boff[kNetLayers];
};
__global__ void k_net_refresh(DimsDev d, long long nparam, const float* th, bf16* wb, bf16* wt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nparam;
       i += (long long)gridDim.x * blockDim.x) {
    int l = -1;
    for (int k = 0; k < kNetLayers; ++k)
      if (i >= d.woff[k] && i < d.boff[k]) l = k;
    if (l < 0) continue;  // bias entries stay FP32
    const bf16 v = __float2bfloat16_rn(th[i]);
    wb[i] = v;
    if (wt) {
      const long long j = i - d.woff[l];
      const int ci = (int)(j % d.cin[l]);
      const long long r = j / d.cin[l];
      const int co = (int)(r % d.cout[l]);
      const int o = (int)(r / d.cout[l]);
      wt[d.woff[l] + ((long long)(26 - o) * d.cin[l] + ci) * d.cout[l] + co] = v;
    }
  }
}

__global__ void k_adam(long long n, float* th, const float* g, float* m, float* v, float lr, float b1, float b2,
                       float eps, float c1, float c2, float gs) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] * gs;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int g_num_sms = 0;
std::mutex g_attr_mu;

int num_sms() {
  if (g_num_sms <= 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms = n > 0 ? n : 1;
  }
  return g_num_sms;
}

ConvArgs conv_base(int n1, int n2, int n3) {
  ConvArgs p{};
  p.n1 = n1;
  p.n2 = n2;
  p.n3 = n3;
  p.V = (long long)n1 * n2 * n3;
  p.ntx = (n1 + TX - 1) / TX;
  p.nty = (n2 + TY - 1) / TY;
  p.ntz = (n3 + TZ - 1) / TZ;
  p.ntiles = (long long)p.ntx * p.nty * p.ntz;
  return p;
}

template <typename K>
void set_smem_attr(K kernel, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_attr_mu);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int CIN, int COUT, int EPI>
void launch_conv(const ConvArgs& p, cudaStream_t st) {
  constexpr size_t sm = conv_smem<CIN, COUT>();
  static std::once_flag once;
  std::call_once(once, [] { set_smem_attr(k_conv<CIN, COUT, EPI>, sm); });
  const long long grid = std::min<long long>(p.ntiles, 2LL * num_sms());
  const int cout_alg = EPI == EPI_WARM || EPI == EPI_LINEAR ? kNetOut : COUT;
  const double fl = 2.0 * 27 * CIN * cout_alg * (double)p.V;
  const double by = (double)p.V * (2.0 * CIN + (EPI == EPI_WARM ? 8.0 * p.c : 2.0 * COUT)) +
                    (EPI == EPI_GRAD ? 2.0 * COUT * p.V : 0.0);
  prof_launch(1, KK_NET_CONV, by, fl, st, [&] { k_conv<CIN, COUT, EPI><<<(int)grid, kThreads, sm, st>>>(p); });
}

template <int CIN, int COUT>
void launch_wgrad(const ConvArgs& p, float* dW, float* db, cudaStream_t st) {
  constexpr size_t sm = wgrad_smem<CIN, COUT>();
  static std::once_flag once;
  std::call_once(once, [] { set_smem_attr(k_conv_wgrad<CIN, COUT>, sm); });
  const long long grid = std::min<long long>(p.ntiles, 4LL * num_sms());
  prof_launch(1, KK_NET_CONV, (double)p.V * 2.0 * (CIN + COUT), 2.0 * 27 * CIN * COUT * (double)p.V, st,
              [&] { k_conv_wgrad<CIN, COUT><<<(int)grid, kThreads, sm, st>>>(p, dW, db); });
}

int aux_blocks(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, kAuxBlocks)); }

// Forward layers run on the tcgen05 kernel where the grid splits into its 8 x 16 tiles
// (wfft_net_conv_kernel(1) selects the mma.sync kernel everywhere, for comparisons).
int g_conv_kernel = 0;
bool tc_grid_ok(const ConvArgs& p) { return g_conv_kernel == 0 && p.n1 % tcconv::TX == 0 && p.n2 % tcconv::TY == 0; }

int* conv_tc_err_ptr() {
  void* q = nullptr;
  return cudaGetSymbolAddress(&q, g_conv_tc_err) == cudaSuccess ? reinterpret_cast<int*>(q) : nullptr;
}

template <int CIN, int COUT, int EPI>
void launch_conv_tc(const ConvArgs& p, cudaStream_t st) {
  constexpr size_t sm = tcconv::Geo<CIN, COUT>::SMEM;
  static std::once_flag once;
  std::call_once(once, [] { set_smem_attr(k_conv_tc<CIN, COUT, EPI>, sm); });
  const long long units = (long long)(p.n1 / tcconv::TX) * (p.n2 / tcconv::TY) * ((p.n3 + tcconv::ZC - 1) / tcconv::ZC);
  const long long grid = std::min<long long>(units, num_sms());
  const int cout_alg = EPI == EPI_WARM || EPI == EPI_LINEAR ? kNetOut : COUT;
  const double fl = 2.0 * 27 * CIN * cout_alg * (double)p.V;
  const double by = (double)p.V * (2.0 * CIN + (EPI == EPI_WARM ? 8.0 * p.c : (EPI == EPI_LINEAR ? 16.0 : 2.0 * COUT)));
  int* err = conv_tc_err_ptr();
  prof_launch(1, KK_NET_CONV, by, fl, st,
              [&] { k_conv_tc<CIN, COUT, EPI><<<(int)grid, tcconv::kThreads, sm, st>>>(p, err); });
}

// Layer l of a network with hidden width H: conv + epilogue.
template <int H>
void layer_fwd(const NetDev& n, int l, ConvArgs p, const bf16* in, void* out, int epi, cudaStream_t st) {
  p.in = in;
  p.W = n.wb + n.d.woff[l];
  p.bias = n.theta + n.d.boff[l];
  p.out = out;
  if constexpr (H == 32) {
    if (tc_grid_ok(p)) {
      if (l == 0) launch_conv_tc<kNetIn, H, EPI_RELU>(p, st);
      else if (l < 3) launch_conv_tc<H, H, EPI_RELU>(p, st);
      else if (epi == EPI_LINEAR) launch_conv_tc<H, kNetOutPad, EPI_LINEAR>(p, st);
      else launch_conv_tc<H, kNetOutPad, EPI_WARM>(p, st);
      return;
    }
  }
  if (l == 0) {
    launch_conv<kNetIn, H, EPI_RELU>(p, st);
  } else if (l < 3) {
    launch_conv<H, H, EPI_RELU>(p, st);
  } else if (epi == EPI_LINEAR) {
    launch_conv<H, kNetOutPad, EPI_LINEAR>(p, st);
  } else {
    launch_conv<H, kNetOutPad, EPI_WARM>(p, st);
  }
}

// Forward through the 4 layers: x -> a1 -> a2 -> a3 -> out (a3 may alias a1).
void net_forward(const NetDev& n, const ConvArgs& base, const bf16* x, bf16* a1, bf16* a2, bf16* a3, int epi,
                 void* out, cudaStream_t st) {
  if (n.d.hidden == 16) {
    layer_fwd<16>(n, 0, base, x, a1, EPI_RELU, st);
    layer_fwd<16>(n, 1, base, a1, a2, EPI_RELU, st);
    layer_fwd<16>(n, 2, base, a2, a3, EPI_RELU, st);
    layer_fwd<16>(n, 3, base, a3, out, epi, st);
  } else {
    layer_fwd<32>(n, 0, base, x, a1, EPI_RELU, st);
    layer_fwd<32>(n, 1, base, a1, a2, EPI_RELU, st);
    layer_fwd<32>(n, 2, base, a2, a3, EPI_RELU, st);
    layer_fwd<32>(n, 3, base, a3, out, epi, st);
  }
}

// Backward from G4 = dL/dy ([V][16]): accumulates dW, db into grad (FP32, parameter layout).
template <int H>
void net_backward_h(const NetDev& n, const ConvArgs& base, const bf16* x, const bf16* a1, const bf16* a2,
                    const bf16* a3, const bf16* g4, bf16* ga, bf16* gb, float* grad, cudaStream_t st) {
  const NetDims& d = n.d;
  ConvArgs p = base;
  // layer 4
  p.in = a3;
  p.gate = g4;
  launch_wgrad<H, kNetOutPad>(p, grad + d.woff[3], grad + d.boff[3], st);
  p = base;
  p.in = g4;
  p.W = n.wt + d.woff[3];
  p.gate = a3;
  p.out = ga;
  launch_conv<kNetOutPad, H, EPI_GRAD>(p, st);
  // layer 3
  p = base;
  p.in = a2;
  p.gate = ga;
  launch_wgrad<H, H>(p, grad + d.woff[2], grad + d.boff[2], st);
  p = base;
  p.in = ga;
  p.W = n.wt + d.woff[2];
  p.gate = a2;
  p.out = gb;
  launch_conv<H, H, EPI_GRAD>(p, st);
  // layer 2
  p = base;
  p.in = a1;
  p.gate = gb;
  launch_wgrad<H, H>(p, grad + d.woff[1], grad + d.boff[1], st);
  p = base;
  p.in = gb;
  p.W = n.wt + d.woff[1];
  p.gate = a1;
  p.out = ga;
  launch_conv<H, H, EPI_GRAD>(p, st);
  // layer 1
  p = base;
  p.in = x;
  p.gate = ga;
  launch_wgrad<kNetIn, H>(p, grad + d.woff[0], grad + d.boff[0], st);
}

void net_backward(const NetDev& n, const ConvArgs& base, const bf16* x, const bf16* a1, const bf16* a2,
                  const bf16* a3, const bf16* g4, bf16* ga, bf16* gb, float* grad, cudaStream_t st) {
  if (n.d.hidden == 16)
    net_backward_h<16>(n, base, x, a1, a2, a3, g4, ga, gb, grad, st);
  else
    net_backward_h<32>(n, base, x, a1, a2, a3, g4, ga, gb, grad, st);
}

void refresh(const NetDev& n, cudaStream_t st) {
  DimsDev dd;
  for (int l = 0; l < kNetLayers; ++l) {
    dd.cin[l] = n.d.cin[l];
    dd.cout[l] = n.d.cout[l];
    dd.woff[l] = (long long)n.d.woff[l];
    dd.boff[l] = (long long)n.d.boff[l];
  }
  prof_launch(1, KK_NET_AUX, 10.0 * n.d.nparam, 0.0, st, [&] {
    k_net_refresh<<<aux_blocks((long long)n.d.nparam), 256, 0, st>>>(dd, (long long)n.d.nparam, n.theta, n.wb, n.wt);
  });
}

template <typename T>
cudaError_t dmalloc(T** p, size_t bytes) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(bytes, 16));
}

}  // namespace

namespace wfft {
// Reads and clears the error word of the tcgen05 convolutions (synchronises the device).
bool net_conv_timed_out() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_conv_tc_err, sizeof(int)) != cudaSuccess) return false;
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_conv_tc_err, &zero, sizeof(int));
  }
  return v != 0;
}
}  // namespace wfft

extern "C" int wfft_net_conv_kernel(int kind) {
  if (kind != 0 && kind != 1) return -1;
  const int prev = g_conv_kernel;
  g_conv_kernel = kind;
  return prev;
}

namespace wfft {

bool net_dims(int hidden, NetDims* d) {
  if (hidden != 16 && hidden != 32) return false;
  NetDims r;
  r.hidden = hidden;
  const int ci[kNetLayers] = {kNetIn, hidden, hidden, hidden};
  const int co[kNetLayers] = {hidden, hidden, hidden, kNetOutPad};
  size_t off = 0;
  for (int l = 0; l < kNetLayers; ++l) {
    r.cin[l] = ci[l];
    r.cout[l] = co[l];
    r.woff[l] = off;
    off += (size_t)27 * ci[l] * co[l];
    r.boff[l] = off;
    off += (size_t)co[l];
  }
  r.nparam = off;
  *d = r;
  return true;
}

size_t net_blob_bytes(int hidden) {
  NetDims d;
  if (!net_dims(hidden, &d)) return 0;
  return sizeof(NetHeader) + d.nparam * sizeof(float);
}

const char* net_parse(const void* blob, size_t bytes, NetDims* d) {
  if (!blob) return "model blob is NULL";
  if (bytes < sizeof(NetHeader)) return "model blob too short";
  NetHeader hd;
  memcpy(&hd, blob, sizeof hd);
  if (hd.magic != kNetMagic) return "not a wfft model blob (magic)";
  if (hd.version != kNetVersion) return "unsupported model blob version";
  if (hd.layers != kNetLayers || hd.cin != kNetIn || hd.cout != kNetOut || hd.cout_pad != kNetOutPad)
    return "unsupported network shape";
  if (!net_dims(hd.hidden, d)) return "hidden width must be 16 or 32";
  if (bytes != sizeof(NetHeader) + d->nparam * sizeof(float)) return "model blob size does not match its header";
  const float* th = reinterpret_cast<const float*>(reinterpret_cast<const char*>(blob) + sizeof(NetHeader));
  for (size_t i = 0; i < d->nparam; ++i) {
    float v;
    memcpy(&v, th + i, sizeof v);
    if (!std::isfinite(v)) return "model parameters are not finite";
  }
  return nullptr;
}

int net_upload(const void* blob, size_t bytes, bool training, NetDev** out, std::string* err) {
  NetDims d;
  if (const char* e = net_parse(blob, bytes, &d)) {
    *err = e;
    return WFFT_EINVAL;
  }
  NetDev* n = new NetDev;
  n->d = d;
  cudaGetDevice(&n->device);
  cudaError_t e = dmalloc(&n->theta, d.nparam * sizeof(float));
  if (e == cudaSuccess) e = dmalloc(&n->wb, d.nparam * sizeof(bf16));
  if (e == cudaSuccess && training) e = dmalloc(&n->wt, d.nparam * sizeof(bf16));
  if (e == cudaSuccess)
    e = cudaMemcpy(n->theta, reinterpret_cast<const char*>(blob) + sizeof(NetHeader), d.nparam * sizeof(float),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    refresh(*n, 0);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    *err = std::string("model upload: ") + cudaGetErrorString(e);
    net_free(n);
    return e == cudaErrorMemoryAllocation ? WFFT_ENOMEM : WFFT_ECUDA;
  }
  *out = n;
  return WFFT_OK;
}

void net_free(NetDev* n) {
  if (!n) return;
  cudaFree(n->theta);
  cudaFree(n->wb);
  cudaFree(n->wt);
  delete n;
}

int net_work_alloc(NetWork* w, long long V, int hidden) {
  if (w->V == V && w->hidden >= hidden && w->x) return WFFT_OK;
  net_work_free(w);
  cudaError_t e = dmalloc(&w->x, (size_t)V * kNetIn * sizeof(bf16));
  if (e == cudaSuccess) e = dmalloc(&w->h0, (size_t)V * hidden * sizeof(bf16));
  if (e == cudaSuccess) e = dmalloc(&w->h1, (size_t)V * hidden * sizeof(bf16));
  if (e == cudaSuccess) e = dmalloc(&w->part, kAuxBlocks * sizeof(double));
  if (e == cudaSuccess) e = dmalloc(&w->scale, 2 * sizeof(float));
  if (e != cudaSuccess) {
    net_work_free(w);
    return e == cudaErrorMemoryAllocation ? WFFT_ENOMEM : WFFT_ECUDA;
  }
  w->V = V;
  w->hidden = hidden;
  return WFFT_OK;
}

void net_work_free(NetWork* w) {
  cudaFree(w->x);
  cudaFree(w->h0);
  cudaFree(w->h1);
  cudaFree(w->part);
  cudaFree(w->scale);
  *w = NetWork{};
}

static void warm_scale_features(NetWork* w, const WarmArgs& a, bool features, cudaStream_t st,
                                float* delta = nullptr) {
  const int nb = aux_blocks(a.V);
  prof_launch(1, KK_NET_AUX, (double)a.V * (a.c * 24.0 + 1.0), (double)a.V * a.c * 8.0, st,
              [&] { k_warm_scale<<<nb, 256, 0, st>>>(a, w->part); });
  prof_launch(1, KK_NET_AUX, 8.0 * nb, 0.0, st,
              [&] { k_warm_scale_fin<<<1, 256, 0, st>>>(w->part, nb, (double)a.c * a.V, w->scale); });
  if (features)
    prof_launch(1, KK_NET_AUX, (double)a.V * (a.c * 28.0 + 4.0 + 32.0), (double)a.V * 40.0, st,
                [&] { k_warm_features<<<nb, 256, 0, st>>>(a, w->scale, w->x, delta); });
}

void net_warm(const NetDev* n, NetWork* w, const WarmArgs& a, float* delta, cudaStream_t st) {
  if (!n) {
    const int nb = aux_blocks((long long)a.c * a.V);
    prof_launch(1, KK_NET_AUX, (double)a.c * a.V * 21.0, 4.0 * a.c * a.V, st,
                [&] { k_warm_taylor<<<nb, 256, 0, st>>>(a, delta); });
    return;
  }
  warm_scale_features(w, a, true, st, delta);
  ConvArgs p = conv_base(a.n1, a.n2, a.n3);
  p.c = a.c;
  p.v = a.v;
  p.a = a.a;
  p.mask = a.mask;
  p.dt = a.dt;
  p.scale = w->scale;
  net_forward(*n, p, w->x, w->h0, w->h1, w->h0, EPI_WARM, delta, st);
}

}  // namespace wfft

// ---------------------------------------------------------------------------
// trainer
// ---------------------------------------------------------------------------
struct wfft_trainer {
  NetDev* net = nullptr;
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  long long adam_t = 0;
  int device = -1;
  cudaStream_t st = nullptr;
  struct Traj {
    int n[3];
    int c;
    long long V;
    uint8_t* mask;
    long long nfree;
  };
  struct Sample {
    int traj;
    bf16* X;
    float* T;
  };
  std::vector<Traj> trajs;
  std::vector<Sample> samples;
  std::vector<void*> allocs;
  long long capV = 0;
  int capH = 0;
  bf16 *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *ga = nullptr, *gb = nullptr, *g4 = nullptr, *xb = nullptr;
  float* Y = nullptr;
  float* Tb = nullptr;
  double* loss = nullptr;
  NetWork work;
  std::string err;
};

static int tfail(wfft_trainer* t, int code, const std::string& msg) {
  if (t)
    t->err = msg;
  else
    set_global_error(msg.c_str());
  return code;
}

#define TCK(t, x)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess)                                                              \
      return tfail(t, e_ == cudaErrorMemoryAllocation ? WFFT_ENOMEM : WFFT_ECUDA,        \
                   std::string(#x) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

static void free_train_buffers(wfft_trainer* t) {
  for (void* p : {(void*)t->a1, (void*)t->a2, (void*)t->a3, (void*)t->ga, (void*)t->gb, (void*)t->g4, (void*)t->xb,
                  (void*)t->Y, (void*)t->Tb})
    cudaFree(p);
  t->a1 = t->a2 = t->a3 = t->ga = t->gb = t->g4 = t->xb = nullptr;
  t->Y = t->Tb = nullptr;
  t->capV = 0;
}

static int ensure_train_buffers(wfft_trainer* t, long long V) {
  const int H = t->net->d.hidden;
  if (V <= t->capV && H <= t->capH) return WFFT_OK;
  free_train_buffers(t);
  TCK(t, dmalloc(&t->a1, (size_t)V * H * sizeof(bf16)));
  TCK(t, dmalloc(&t->a2, (size_t)V * H * sizeof(bf16)));
  TCK(t, dmalloc(&t->a3, (size_t)V * H * sizeof(bf16)));
  TCK(t, dmalloc(&t->ga, (size_t)V * H * sizeof(bf16)));
  TCK(t, dmalloc(&t->gb, (size_t)V * H * sizeof(bf16)));
  TCK(t, dmalloc(&t->g4, (size_t)V * kNetOutPad * sizeof(bf16)));
  TCK(t, dmalloc(&t->xb, (size_t)V * kNetIn * sizeof(bf16)));
  TCK(t, dmalloc(&t->Y, (size_t)V * 4 * sizeof(float)));
  TCK(t, dmalloc(&t->Tb, (size_t)V * 4 * sizeof(float)));
  t->capV = V;
  t->capH = H;
  return WFFT_OK;
}

// One forward + backward of a sample; accumulates its gradient into t->grad and its
// loss sum into *t->loss.  gs = d(loss)/d(sum of squares).
static void sample_fwd_bwd(wfft_trainer* t, const int n[3], int c, const bf16* X, const float* T,
                           const uint8_t* mask, float gs, cudaStream_t st) {
  ConvArgs p = conv_base(n[0], n[1], n[2]);
  net_forward(*t->net, p, X, t->a1, t->a2, t->a3, EPI_LINEAR, t->Y, st);
  const long long V = p.V;
  prof_launch(1, KK_NET_AUX, (double)V * (32.0 + 32.0 + 1.0), 3.0 * V, st, [&] {
    k_loss_grad<<<aux_blocks(V), 256, 0, st>>>(V, c, t->Y, T, mask, gs, t->g4, t->loss);
  });
  net_backward(*t->net, p, X, t->a1, t->a2, t->a3, t->g4, t->ga, t->gb, t->grad, st);
}

static int trainer_init_opt(wfft_trainer* t) {
  const size_t np = t->net->d.nparam;
  TCK(t, dmalloc(&t->grad, np * sizeof(float)));
  TCK(t, dmalloc(&t->m, np * sizeof(float)));
  TCK(t, dmalloc(&t->v, np * sizeof(float)));
  TCK(t, cudaMemset(t->grad, 0, np * sizeof(float)));
  TCK(t, cudaMemset(t->m, 0, np * sizeof(float)));
  TCK(t, cudaMemset(t->v, 0, np * sizeof(float)));
  TCK(t, dmalloc(&t->loss, sizeof(double)));
  return WFFT_OK;
}

extern "C" size_t wfft_model_bytes(int hidden) { return net_blob_bytes(hidden); }

extern "C" int wfft_model_init(int hidden, unsigned long long seed, void* blob, size_t bytes) {
  NetDims d;
  if (!net_dims(hidden, &d)) return tfail(nullptr, WFFT_EINVAL, "hidden width must be 16 or 32");
  if (!blob || bytes != net_blob_bytes(hidden)) return tfail(nullptr, WFFT_EINVAL, "blob size must be wfft_model_bytes(hidden)");
  NetHeader hd{kNetMagic, kNetVersion, kNetLayers, kNetIn, hidden, kNetOut, kNetOutPad, 0};
  std::vector<float> th(d.nparam, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  // He-normal weights for the ReLU layers; the output layer starts at zero, so an
  // untrained network predicts exactly the Taylor increment
  for (int l = 0; l < kNetLayers - 1; ++l) {
    const double sd = std::sqrt(2.0 / (27.0 * d.cin[l]));
    for (size_t i = 0; i < (size_t)27 * d.cin[l] * d.cout[l]; ++i) th[d.woff[l] + i] = (float)(sd * nd(rng));
  }
  memcpy(blob, &hd, sizeof hd);
  memcpy(reinterpret_cast<char*>(blob) + sizeof hd, th.data(), th.size() * sizeof(float));
  return WFFT_OK;
}

extern "C" int wfft_trainer_create(const void* blob, size_t bytes, void* cuda_stream, wfft_trainer** out) {
  if (!out) return tfail(nullptr, WFFT_EINVAL, "out is NULL");
  *out = nullptr;
  NetDims d;
  if (const char* e = net_parse(blob, bytes, &d)) return tfail(nullptr, WFFT_EINVAL, e);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return tfail(nullptr, WFFT_ECUDA, "no CUDA device");
  }
  wfft_trainer* t = new wfft_trainer;
  t->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&t->device);
  std::string err;
  int rc = net_upload(blob, bytes, true, &t->net, &err);
  if (rc == WFFT_OK) rc = trainer_init_opt(t);
  else t->err = err;
  if (rc != WFFT_OK) {
    std::string m = t->err;
    wfft_trainer_destroy(t);
    return tfail(nullptr, rc, m);
  }
  *out = t;
  return WFFT_OK;
}

extern "C" void wfft_trainer_destroy(wfft_trainer* t) {
  if (!t) return;
  if (t->st) cudaStreamSynchronize(t->st);
  cudaDeviceSynchronize();
  free_train_buffers(t);
  net_work_free(&t->work);
  for (void* p : t->allocs) cudaFree(p);
  cudaFree(t->grad);
  cudaFree(t->m);
  cudaFree(t->v);
  cudaFree(t->loss);
  net_free(t->net);
  delete t;
}

extern "C" long long wfft_trainer_samples(const wfft_trainer* t) { return t ? (long long)t->samples.size() : -1; }

extern "C" const char* wfft_trainer_error(const wfft_trainer* t) { return t ? t->err.c_str() : ""; }

extern "C" int wfft_trainer_collect(wfft_trainer* t, wfft_handle* h, const double* U, int nsteps,
                                    wfft_step_info* infos) {
  if (!t) return tfail(nullptr, WFFT_EINVAL, "null trainer");
  if (!h || !U || nsteps < 0) return tfail(t, WFFT_EINVAL, "handle and U are required, nsteps >= 0");
  if (nsteps == 0) return WFFT_OK;
  WarmArgs a;
  cudaStream_t st;
  int dev;
  if (handle_warm_args(h, U, &a, &st, &dev) != WFFT_OK) return tfail(t, WFFT_EINVAL, "invalid handle");
  if (dev != t->device) return tfail(t, WFFT_EINVAL, "handle and trainer are on different devices");
  const long long V = a.V;
  int rc = net_work_alloc(&t->work, V, 16);
  if (rc) return tfail(t, rc, "warm-start work buffers");
  // per trajectory: the component mask; per step: features, target
  wfft_trainer::Traj tr{{a.n1, a.n2, a.n3}, a.c, V, nullptr, 0};
  if (a.mask) {
    TCK(t, dmalloc(&tr.mask, (size_t)V));
    t->allocs.push_back(tr.mask);
    TCK(t, cudaMemcpyAsync(tr.mask, a.mask, (size_t)V, cudaMemcpyDeviceToDevice, st));
    std::vector<uint8_t> hm((size_t)V);
    TCK(t, cudaMemcpyAsync(hm.data(), a.mask, (size_t)V, cudaMemcpyDeviceToHost, st));
    TCK(t, cudaStreamSynchronize(st));
    long long fixed = 0;
    for (long long i = 0; i < V; ++i)
      for (int k = 0; k < a.c; ++k) fixed += (hm[i] >> k) & 1;
    tr.nfree = (long long)a.c * V - fixed;
  } else {
    tr.nfree = (long long)a.c * V;
  }
  const int ti = (int)t->trajs.size();
  t->trajs.push_back(tr);
  const size_t xb = (size_t)V * kNetIn * sizeof(bf16), tb = (size_t)V * 4 * sizeof(float);
  char* pool;
  TCK(t, dmalloc(&pool, (size_t)nsteps * (xb + tb)));
  t->allocs.push_back(pool);
  double* a_old;
  TCK(t, dmalloc(&a_old, (size_t)a.c * V * sizeof(double)));
  for (int i = 0; i < nsteps; ++i) {
    handle_warm_args(h, U + 3 * i, &a, &st, &dev);
    bf16* X = reinterpret_cast<bf16*>(pool + (size_t)i * (xb + tb));
    float* T = reinterpret_cast<float*>(pool + (size_t)i * (xb + tb) + xb);
    warm_scale_features(&t->work, a, true, st);
    cudaMemcpyAsync(X, t->work.x, xb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a_old, a.a, (size_t)a.c * V * sizeof(double), cudaMemcpyDeviceToDevice, st);
    wfft_step_info info;
    rc = wfft_step(h, U + 3 * i, &info);
    if (infos) infos[i] = info;
    if (rc != WFFT_OK) {
      cudaFree(a_old);
      return tfail(t, rc, std::string("solver step failed: ") + wfft_last_error(h));
    }
    k_net_target<<<aux_blocks(V), 256, 0, st>>>(V, a.c, a.a, a_old, a.mask, a.theta, t->work.scale, T);
    t->samples.push_back({ti, X, T});
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(a_old);
  TCK(t, e);
  TCK(t, cudaGetLastError());
  return WFFT_OK;
}

extern "C" int wfft_trainer_fit(wfft_trainer* t, int epochs, int batch, double lr, unsigned long long seed,
                                double* loss_out) {
  if (!t) return tfail(nullptr, WFFT_EINVAL, "null trainer");
  if (epochs < 0 || batch < 1 || !(lr > 0)) return tfail(t, WFFT_EINVAL, "epochs >= 0, batch >= 1, lr > 0");
  if (t->samples.empty()) return tfail(t, WFFT_EINVAL, "no samples collected");
  long long maxV = 0;
  for (const auto& tr : t->trajs) maxV = std::max(maxV, tr.V);
  int rc = ensure_train_buffers(t, maxV);
  if (rc) return rc;
  cudaStream_t st = t->st;
  std::mt19937_64 rng(seed);
  std::vector<int> order(t->samples.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  const size_t np = t->net->d.nparam;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    TCK(t, cudaMemsetAsync(t->loss, 0, sizeof(double), st));
    int inb = 0;
    for (size_t k = 0; k < order.size(); ++k) {
      const auto& s = t->samples[order[k]];
      const auto& tr = t->trajs[s.traj];
      const float gs = tr.nfree > 0 ? (float)(2.0 / (double)tr.nfree) : 0.f;
      sample_fwd_bwd(t, tr.n, tr.c, s.X, s.T, tr.mask, gs, st);
      if (++inb == batch || k + 1 == order.size()) {
        ++t->adam_t;
        const float c1 = 1.f / (1.f - std::pow(b1, (float)t->adam_t));
        const float c2 = 1.f / (1.f - std::pow(b2, (float)t->adam_t));
        const float gsc = 1.f / (float)inb;
        prof_launch(1, KK_NET_AUX, 20.0 * np, 10.0 * np, st, [&] {
          k_adam<<<aux_blocks((long long)np), 256, 0, st>>>((long long)np, t->net->theta, t->grad, t->m, t->v,
                                                             (float)lr, b1, b2, eps, c1, c2, gsc);
        });
        TCK(t, cudaMemsetAsync(t->grad, 0, np * sizeof(float), st));
        refresh(*t->net, st);
        inb = 0;
      }
    }
    double ls = 0.0;
    TCK(t, cudaMemcpyAsync(&ls, t->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    TCK(t, cudaStreamSynchronize(st));
    // mean over samples of the per-sample mean squared error
    double nf = 0.0;
    for (const auto& s : t->samples) nf += (double)t->trajs[s.traj].nfree;
    last = nf > 0 ? ls / nf : 0.0;
  }
  TCK(t, cudaGetLastError());
  if (net_conv_timed_out()) return tfail(t, WFFT_ETIMEOUT, "a tensor-core convolution's wait expired");
  if (loss_out) *loss_out = last;
  return WFFT_OK;
}

extern "C" int wfft_trainer_get_model(const wfft_trainer* t, void* blob, size_t bytes) {
  if (!t || !blob) return tfail(nullptr, WFFT_EINVAL, "trainer and blob are required");
  const NetDims& d = t->net->d;
  if (bytes != net_blob_bytes(d.hidden)) return tfail(nullptr, WFFT_EINVAL, "blob size does not match the model");
  NetHeader hd{kNetMagic, kNetVersion, kNetLayers, kNetIn, d.hidden, kNetOut, kNetOutPad, 0};
  memcpy(blob, &hd, sizeof hd);
  if (t->st) cudaStreamSynchronize(t->st);
  cudaError_t e = cudaMemcpy(reinterpret_cast<char*>(blob) + sizeof hd, t->net->theta, d.nparam * sizeof(float),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return tfail(nullptr, WFFT_ECUDA, cudaGetErrorString(e));
  return WFFT_OK;
}

// ---------------------------------------------------------------------------
// single-call network evaluation (host buffers), for testing against a reference
// ---------------------------------------------------------------------------
static int check_grid(const int n[3], long long* V) {
  if (!n || n[0] < 1 || n[1] < 1 || n[2] < 1) return WFFT_EINVAL;
  *V = (long long)n[0] * n[1] * n[2];
  return WFFT_OK;
}

extern "C" int wfft_net_forward(const void* blob, size_t bytes, const int n[3], const float* x, float* y) {
  long long V;
  if (check_grid(n, &V) || !x || !y) return tfail(nullptr, WFFT_EINVAL, "grid, x and y are required");
  wfft_trainer* t = nullptr;
  int rc = wfft_trainer_create(blob, bytes, nullptr, &t);
  if (rc) return rc;
  rc = ensure_train_buffers(t, V);
  float* xf = nullptr;
  if (rc == WFFT_OK && dmalloc(&xf, (size_t)V * kNetIn * sizeof(float)) != cudaSuccess) rc = WFFT_ENOMEM;
  if (rc == WFFT_OK) {
    cudaMemcpy(xf, x, (size_t)V * kNetIn * sizeof(float), cudaMemcpyHostToDevice);
    k_f32_to_bf16<<<aux_blocks(V * kNetIn), 256>>>(xf, t->xb, V * kNetIn);
    ConvArgs p = conv_base(n[0], n[1], n[2]);
    net_forward(*t->net, p, t->xb, t->a1, t->a2, t->a3, EPI_LINEAR, t->Y, 0);
    std::vector<float> y4((size_t)V * 4);
    cudaError_t e = cudaMemcpy(y4.data(), t->Y, y4.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = tfail(nullptr, WFFT_ECUDA, cudaGetErrorString(e));
    } else if (net_conv_timed_out()) {
      rc = tfail(nullptr, WFFT_ETIMEOUT, "a tensor-core convolution's wait expired");
    } else {
      for (long long i = 0; i < V; ++i)
        for (int k = 0; k < kNetOut; ++k) y[i * kNetOut + k] = y4[i * 4 + k];
    }
  }
  cudaFree(xf);
  wfft_trainer_destroy(t);
  return rc;
}

extern "C" int wfft_net_loss_grad(const void* blob, size_t bytes, const int n[3], int c, const float* x,
                                  const float* target, const unsigned char* mask, float* grad, double* loss) {
  long long V;
  if (check_grid(n, &V) || !x || !target || !grad || c < 1 || c > 3)
    return tfail(nullptr, WFFT_EINVAL, "grid, x, target, grad required; 1 <= c <= 3");
  wfft_trainer* t = nullptr;
  int rc = wfft_trainer_create(blob, bytes, nullptr, &t);
  if (rc) return rc;
  rc = ensure_train_buffers(t, V);
  float* xf = nullptr;
  uint8_t* dm = nullptr;
  long long nfree = (long long)c * V;
  if (rc == WFFT_OK && dmalloc(&xf, (size_t)V * kNetIn * sizeof(float)) != cudaSuccess) rc = WFFT_ENOMEM;
  if (rc == WFFT_OK && mask) {
    if (dmalloc(&dm, (size_t)V) != cudaSuccess) rc = WFFT_ENOMEM;
    else {
      cudaMemcpy(dm, mask, (size_t)V, cudaMemcpyHostToDevice);
      for (long long i = 0; i < V; ++i)
        for (int k = 0; k < c; ++k) nfree -= (mask[i] >> k) & 1;
    }
  }
  if (rc == WFFT_OK) {
    std::vector<float> t4((size_t)V * 4, 0.f);
    for (long long i = 0; i < V; ++i)
      for (int k = 0; k < c; ++k) t4[i * 4 + k] = target[i * 3 + k];
    cudaMemcpy(t->Tb, t4.data(), t4.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(xf, x, (size_t)V * kNetIn * sizeof(float), cudaMemcpyHostToDevice);
    k_f32_to_bf16<<<aux_blocks(V * kNetIn), 256>>>(xf, t->xb, V * kNetIn);
    cudaMemset(t->loss, 0, sizeof(double));
    const float gs = nfree > 0 ? (float)(2.0 / (double)nfree) : 0.f;
    sample_fwd_bwd(t, n, c, t->xb, t->Tb, dm, gs, 0);
    double ls = 0;
    cudaError_t e = cudaMemcpy(&ls, t->loss, sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(grad, t->grad, t->net->d.nparam * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) rc = tfail(nullptr, WFFT_ECUDA, cudaGetErrorString(e));
    else if (loss) *loss = nfree > 0 ? ls / (double)nfree : 0.0;
  }
  cudaFree(xf);
  cudaFree(dm);
  wfft_trainer_destroy(t);
  return rc;
}
