// Column passes over a 256-point axis as two radix-16 stages held in registers
// (FP32, 3-D grids).
//
// The transform is the DFT of Sec. 2.1.3 (Eq. Fourier_derivatives) along y or z,
// written for N = 256 = 16 x 16.  With n = j + 16 r and k = ka + 16 kb,
//   X[ka + 16 kb] = sum_j W16^(j kb) [ W256^(j ka) sum_r x[j + 16 r] W16^(r ka) ]
// (W_M = exp(-2 pi i / M), conjugated for the inverse).  A block owns BXC = 4, 8 or 16
// consecutive kx columns (32-, 64- or 128-byte rows of FP32 complex) x the 256 points
// of the axis, 16 BXC threads; thread (b = t % BXC, j = t / BXC) loads the 16 points
// j + 16 r of column b straight from
// global memory, takes the first 16-point DFT and the twiddles in registers and
// writes one transposition buffer in shared memory; after a barrier thread (b, ka)
// reads its 16 values, takes the second DFT and holds X[ka + 16 kb], kb = 0..15, in
// registers.  The pointwise work of the method runs on those registers, and the
// inverse runs the same two stages in the opposite order (first over kb, twiddles,
// transposition, then over ka), so that thread (b, m1) ends with x[m1 + 16 m2] and
// stores it straight to global memory.  Each element crosses shared memory twice per
// transform (one write, one read), against a load, a store and two stage round trips
// in the general column kernels, and all index arithmetic is compile-time.  The
// twiddles W256^(j k) are one 256-entry table per block (sincospif of j k / 128).
//
// Passes (one block per BXC-column tile; `axis` is 1 (y) or 2 (z)):
//   k_col256<OP_FWD / OP_INV>: plain transform of component blockIdx.y
//   k_col256<OP_GRAD>: u^ -> engineering strains e^ = (i/V) B(xi) u^ (Eq. Fourier_ND_A)
//   k_col256<OP_DIV>:  sigma^ -> t^ = (-theta/V) i B(xi)^T sigma^
//   k_col256<OP_PREC>: r^ -> z^ = (1/V)(theta K(xi) + rho_bar I)^-1 r^ (Eq. precond),
//                      with the Parseval partial sum of (r, z)
// The fused passes hold three components (48 complex values per thread) in registers
// and use three transposition buffers; the six-slot sides (strains, stresses) go
// through them as two rounds of three.
#pragma once
#include "passes.cuh"

namespace wfft {

// Row stride (complex elements) of a transposition buffer of BXC columns: 16 BXC plus a
// pad for 4- and 8-column tiles, so that the second stage's reads (BXC columns x 32/BXC
// rows per warp) spread over all banks.
__host__ __device__ __forceinline__ constexpr int col256_rs(int bxc) { return 16 * bxc + (bxc == 16 ? 0 : bxc); }
// Shared memory of a k_col256 pass: the twiddle table and nbuf transposition buffers.
__host__ __device__ __forceinline__ constexpr size_t col256_smem(int nbuf, int bxc) {
  return (size_t)(256 + nbuf * 16 * col256_rs(bxc)) * sizeof(float2);
}

namespace c256 {

using F2 = float2;

// transposition buffer element (row, col) of column b: rows are the 16 values a
// thread of the second stage reads; a warp's writes touch 256 consecutive bytes
template <int BXC>
__device__ __forceinline__ int sidx(int row, int col, int b) { return row * col256_rs(BXC) + col * BXC + b; }

// first stage of a forward (SG = -1) or inverse (SG = +1) transform: v holds
// x[j + 16 r] (r = 0..15); leaves W^(SG j ka) DFT_16(v)[ka] in buffer row ka, column j
template <int SG, int BXC>
__device__ __forceinline__ void stage1(F2 (&v)[16], int j, int b, const F2* tw, F2* buf) {
  Dft<float, 16>::run(v, SG, nullptr, 0);
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    F2 w = tw[k * 16 + j];  // W256^(j k), row k of the table
    if (SG > 0) w.y = -w.y;
    v[k] = cmul<float>(v[k], w);
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) buf[sidx<BXC>(k, j, b)] = v[k];
}

// second stage: thread row ka reads its 16 values and leaves X[ka + 16 kb] in v[kb]
template <int SG, int BXC>
__device__ __forceinline__ void stage2(F2 (&v)[16], int ka, int b, const F2* buf) {
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = buf[sidx<BXC>(ka, i, b)];
  Dft<float, 16>::run(v, SG, nullptr, 0);
}

// the 16 points of a thread, 16 axis elements apart (est16 elements; a 256-point axis
// of a spectral component spans less than 2^31 elements)
__device__ __forceinline__ void gload(F2 (&v)[16], const F2* p, int est16, bool ok) {
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = ok ? p[r * est16] : cmake<float>(0.f, 0.f);
}

__device__ __forceinline__ void gstore(const F2 (&v)[16], F2* p, int est16, bool ok) {
  if (!ok) return;
#pragma unroll
  for (int r = 0; r < 16; ++r) p[r * est16] = v[r];
}

}  // namespace c256

// Blocks per SM the fused passes are compiled for (registers per thread follow): three
// 128-thread blocks (at most 170 registers) over 8-column tiles, one block otherwise.
// Measured at 256^3: the gradient and preconditioner passes take 0.22 / 0.19 ms with three
// blocks against 0.26 / 0.22 ms with two (255 registers); at 128 registers every fused
// pass spills and runs 20-45 % slower.
__host__ __device__ constexpr int col256_fused_minb(int op, int bxc) {
  return (bxc == 8 && op >= OP_GRAD) ? 3 : 1;
}

template <int OP, int BXC, int BATCH>
__global__ void __launch_bounds__(16 * BXC, (OP == OP_FWD || OP == OP_INV) ? 64 / BXC : col256_fused_minb(OP, BXC))
    k_col256(const Desc<float>* __restrict__ dd, BatchArgs<float> ba, int axis) {
  using namespace c256;
  int blk;
  const Desc<float>* __restrict__ Dp = pick_ptr<float, BATCH>(dd, ba, blk);
  const Desc<float>& D = *Dp;
  if (D.sc->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  F2* tw = reinterpret_cast<F2*>(smraw);
  F2* S = tw + 256;
  constexpr int kBuf = 16 * col256_rs(BXC);
  const ColGeo<float> g = col_geo<float>(D, axis, BXC, blk);
  const int t = threadIdx.x;
  const int b = t % BXC, j = t / BXC;
  // twiddle table by stage-1 output k (row) and thread j (column): entry 16 k + j holds
  // W256^(j k), so the 16 threads of a row read 16 consecutive entries (no bank conflicts)
  for (int m = t; m < 256; m += 16 * BXC) {
    float s, c;
    sincospif((float)((m >> 4) * (m & 15)) * (1.0f / 128.0f), &s, &c);
    tw[m] = cmake<float>(c, -s);
  }
  const bool ok = g.kx0 + b < D.nh;
  const long long est = g.est;
  const int est16 = (int)(16 * est);
  // element offset of this thread's first point (j) of column b; the stride between its
  // 16 points is 16 est
  const long long off = g.base + (long long)j * est + b;
  F2 v[16];
  __syncthreads();

  if constexpr (OP == OP_FWD || OP == OP_INV) {
    constexpr int SG = OP == OP_FWD ? -1 : +1;
    F2* p = D.spec + (long long)blockIdx.y * D.Vh + off;
    gload(v, p, est16, ok);
    stage1<SG, BXC>(v, j, b, tw, S);
    __syncthreads();
    stage2<SG, BXC>(v, j, b, S);
    gstore(v, p, est16, ok);
  } else {
    // frequency of the three axes for element k of this thread's column
    auto xi3 = [&](int k, float& x1, float& x2, float& x3) { col_xi<float>(D, g, axis, k, b, x1, x2, x3); };
    if constexpr (OP == OP_PREC) {
      F2 R[3][16];
      // all three components' loads in flight before the first transform
#pragma unroll
      for (int c = 0; c < 3; ++c) gload(R[c], D.spec + c * D.Vh + off, est16, ok);
#pragma unroll
      for (int c = 0; c < 3; ++c) stage1<-1, BXC>(R[c], j, b, tw, S + c * kBuf);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 3; ++c) stage2<-1, BXC>(R[c], j, b, S + c * kBuf);
      const int kx = g.kx0 + b;
      const float wgt = !ok ? 0.f : ((kx == 0 || 2 * kx == D.n1) ? 1.f : 2.f);
      DotAcc<float> acc;
      const float iv = D.invV;
#pragma unroll
      for (int kb = 0; kb < 16; ++kb) {
        float x1, x2, x3;
        xi3(j + 16 * kb, x1, x2, x3);
        const float m0 = x1 * x1, m1 = x2 * x2, m2 = x3 * x3, m3 = x2 * x3, m4 = x1 * x3, m5 = x1 * x2;
        float Mv[6];
#pragma unroll
        for (int pr = 0; pr < 6; ++pr)
          Mv[pr] = D.kq[pr][0] * m0 + D.kq[pr][1] * m1 + D.kq[pr][2] * m2 + D.kq[pr][3] * m3 + D.kq[pr][4] * m4 +
                   D.kq[pr][5] * m5;
        const float a = Mv[0] + D.rhobar, bb = Mv[1] + D.rhobar, cc = Mv[2] + D.rhobar, f = Mv[3], ee = Mv[4],
                    d = Mv[5];
        const float A00 = bb * cc - f * f, A11 = a * cc - ee * ee, A22 = a * bb - d * d;
        const float A01 = ee * f - d * cc, A02 = d * f - bb * ee, A12 = d * ee - a * f;
        const float det = a * A00 + d * A01 + ee * A02;
        const float id = iv / det;
        const F2 r1 = R[0][kb], r2 = R[1][kb], r3 = R[2][kb];
        const F2 z1 = cscale<float>(cadd<float>(cadd<float>(cscale<float>(r1, A00), cscale<float>(r2, A01)),
                                                cscale<float>(r3, A02)), id);
        const F2 z2 = cscale<float>(cadd<float>(cadd<float>(cscale<float>(r1, A01), cscale<float>(r2, A11)),
                                                cscale<float>(r3, A12)), id);
        const F2 z3 = cscale<float>(cadd<float>(cadd<float>(cscale<float>(r1, A02), cscale<float>(r2, A12)),
                                                cscale<float>(r3, A22)), id);
        acc.add_prod(wgt * r1.x, z1.x);
        acc.add_prod(wgt * r1.y, z1.y);
        acc.add_prod(wgt * r2.x, z2.x);
        acc.add_prod(wgt * r2.y, z2.y);
        acc.add_prod(wgt * r3.x, z3.x);
        acc.add_prod(wgt * r3.y, z3.y);
        R[0][kb] = z1;
        R[1][kb] = z2;
        R[2][kb] = z3;
      }
      // every thread has read its rows of the buffers (the sum's barriers) before the
      // inverse's first stage overwrites them
      const double s = block_sum(acc.value());
      if (t == 0) D.part[PT_B][blk] = s;
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 3; ++c) stage1<+1, BXC>(R[c], j, b, tw, S + c * kBuf);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        stage2<+1, BXC>(v, j, b, S + c * kBuf);
        gstore(v, D.spec + c * D.Vh + off, est16, ok);
      }
    } else if constexpr (OP == OP_GRAD) {
      F2 U[3][16];
#pragma unroll
      for (int c = 0; c < 3; ++c) gload(U[c], D.spec + c * D.Vh + off, est16, ok);
#pragma unroll
      for (int c = 0; c < 3; ++c) stage1<-1, BXC>(U[c], j, b, tw, S + c * kBuf);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 3; ++c) stage2<-1, BXC>(U[c], j, b, S + c * kBuf);
      __syncthreads();
      const float iv = D.invV;
      // round 0: gamma_11, gamma_12, gamma_13 (slots 0, 5, 4: every term with u1)
      // round 1: gamma_22, gamma_33, gamma_23 (slots 1, 2, 3)
#pragma unroll
      for (int round = 0; round < 2; ++round) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
          for (int kb = 0; kb < 16; ++kb) {
            float x1, x2, x3;
            xi3(j + 16 * kb, x1, x2, x3);
            F2 e;
            if (round == 0) {
              if (q == 0) e = cscale<float>(U[0][kb], x1);
              else if (q == 1) e = cadd<float>(cscale<float>(U[1][kb], x1), cscale<float>(U[0][kb], x2));
              else e = cadd<float>(cscale<float>(U[2][kb], x1), cscale<float>(U[0][kb], x3));
            } else {
              if (q == 0) e = cscale<float>(U[1][kb], x2);
              else if (q == 1) e = cscale<float>(U[2][kb], x3);
              else e = cadd<float>(cscale<float>(U[2][kb], x2), cscale<float>(U[1][kb], x3));
            }
            v[kb] = cmuli<float>(cscale<float>(e, iv), +1);
          }
          stage1<+1, BXC>(v, j, b, tw, S + q * kBuf);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int slot = round == 0 ? (q == 0 ? 0 : q == 1 ? 5 : 4) : (q == 0 ? 1 : q == 1 ? 2 : 3);
          stage2<+1, BXC>(v, j, b, S + q * kBuf);
          gstore(v, D.spec + slot * D.Vh + off, est16, ok);
        }
        __syncthreads();
      }
    } else {  // OP_DIV
      // t_i = sum_j xi_j sigma_ij, one output completed per round so that at most two
      // accumulators stay live while stresses load: round 0 reads s11, s12, s13 (t_1
      // complete), round 1 s22, s23 (t_2), round 2 s33 (t_3); a completed t_i takes its
      // first inverse stage into buffer i at once (spectral components: 11, 22, 33, 23, 13, 12)
      const float f = D.mthetaInvV;
      F2 t2[16], t3[16];
      auto finish = [&](F2 (&tv)[16], int c) {
#pragma unroll
        for (int kb = 0; kb < 16; ++kb) tv[kb] = cmuli<float>(cscale<float>(tv[kb], f), +1);
        stage1<+1, BXC>(tv, j, b, tw, S + c * kBuf);
      };
      {
        F2 in[3][16];
        gload(in[0], D.spec + 0 * D.Vh + off, est16, ok);  // s11
        gload(in[1], D.spec + 5 * D.Vh + off, est16, ok);  // s12
        gload(in[2], D.spec + 4 * D.Vh + off, est16, ok);  // s13
#pragma unroll
        for (int q = 0; q < 3; ++q) stage1<-1, BXC>(in[q], j, b, tw, S + q * kBuf);
        __syncthreads();
        F2 t1[16];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          stage2<-1, BXC>(v, j, b, S + q * kBuf);
#pragma unroll
          for (int kb = 0; kb < 16; ++kb) {
            float x1, x2, x3;
            xi3(j + 16 * kb, x1, x2, x3);
            const F2 sg = v[kb];
            if (q == 0) {
              t1[kb] = cscale<float>(sg, x1);
            } else if (q == 1) {  // s12
              t1[kb] = cadd<float>(t1[kb], cscale<float>(sg, x2));
              t2[kb] = cscale<float>(sg, x1);
            } else {  // s13
              t1[kb] = cadd<float>(t1[kb], cscale<float>(sg, x3));
              t3[kb] = cscale<float>(sg, x1);
            }
          }
        }
        __syncthreads();
        finish(t1, 0);
      }
      {
        F2 in[2][16];
        gload(in[0], D.spec + 1 * D.Vh + off, est16, ok);  // s22
        gload(in[1], D.spec + 3 * D.Vh + off, est16, ok);  // s23
#pragma unroll
        for (int q = 0; q < 2; ++q) stage1<-1, BXC>(in[q], j, b, tw, S + (q + 1) * kBuf);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          stage2<-1, BXC>(v, j, b, S + (q + 1) * kBuf);
#pragma unroll
          for (int kb = 0; kb < 16; ++kb) {
            float x1, x2, x3;
            xi3(j + 16 * kb, x1, x2, x3);
            const F2 sg = v[kb];
            if (q == 0) {
              t2[kb] = cadd<float>(t2[kb], cscale<float>(sg, x2));
            } else {  // s23
              t2[kb] = cadd<float>(t2[kb], cscale<float>(sg, x3));
              t3[kb] = cadd<float>(t3[kb], cscale<float>(sg, x2));
            }
          }
        }
        __syncthreads();
        finish(t2, 1);
      }
      gload(v, D.spec + 2 * D.Vh + off, est16, ok);  // s33
      stage1<-1, BXC>(v, j, b, tw, S + 2 * kBuf);
      __syncthreads();
      stage2<-1, BXC>(v, j, b, S + 2 * kBuf);
#pragma unroll
      for (int kb = 0; kb < 16; ++kb) {
        float x1, x2, x3;
        xi3(j + 16 * kb, x1, x2, x3);
        t3[kb] = cadd<float>(t3[kb], cscale<float>(v[kb], x3));
      }
      __syncthreads();
      finish(t3, 2);
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        stage2<+1, BXC>(v, j, b, S + c * kBuf);
        gstore(v, D.spec + c * D.Vh + off, est16, ok);
      }
    }
  }
}

}  // namespace wfft
