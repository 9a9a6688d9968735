// x passes over 256-point rows with register-held radix-16 stages (FP32, 3-D grids).
//
// Two real lines are transformed as one complex line Z = a + i b (Sec. 2.1.3, the
// real-data form of Eq. Fourier_derivatives); its 256-point DFT is taken as two
// 16-point stages as in the register-stage column kernels: thread (pair, j) holds
// Z[j + 16 r] (r = 0..15), takes the first DFT and the twiddles W256^(j k) in registers
// and writes the pair's transposition buffer; after a barrier thread (pair, ka) reads its
// row and ends with Z[ka + 16 kb] (forward) or z[ka + 16 kb] (inverse).  So an inverse
// transform leaves each thread the real values of its two lines at x = ka + 16 kb, the
// positions its next forward transform starts from: pointwise work between an inverse
// and a forward transform needs no exchange (the Hooke step does, because the six
// strains of a voxel sit in three threads).  Half spectra are read straight from
// global memory (Z_k = A_k + i B_k, Z_{256-k} = conj A_k + i conj B_k) and written
// from a natural-order copy of Z (A_k = (Z_k + conj Z_{256-k}) / 2,
// B_k = (Z_k - conj Z_{256-k}) / 2i).  Real rows are read and written 16 elements
// apart per thread (64-byte runs per line and warp access).
//
// Kernels (one block per LX lines, as the general x passes, so the partial-sum arrays
// keep their block count):
//   k_xmid256: strain half spectra -> strains -> sigma = C(x):e -> stress half spectra
//   k_xinv256<POST_APPLY>: q = t + rho p, mask, (p, q)
//   k_xinv256<POST_PREC_PUPD>: z = P(t), p = z + beta p, half spectrum of p
//   k_xfwd256<PRE_RUPD>: d += alpha p, r -= alpha q, ||r||^2, half spectrum of r
#pragma once
#include "passes.cuh"

namespace wfft {

namespace x256 {

using F2 = float2;
// a pair's transposition buffer: 16 rows of 16 complex values, row stride 17 (the
// second stage's reads of 16 rows per half-warp then fall on distinct banks)
constexpr int kRS = 17;
constexpr int kPairBuf = 16 * kRS;  // >= 256: also holds a natural-order line

template <int SG>
__device__ __forceinline__ void stage1(F2 (&v)[16], int j, const F2* tw, F2* buf) {
  Dft<float, 16>::run(v, SG, nullptr, 0);
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    F2 w = tw[k * 16 + j];  // W256^(j k), row k of the table
    if (SG > 0) w.y = -w.y;
    v[k] = cmul<float>(v[k], w);
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) buf[k * kRS + j] = v[k];
}

template <int SG>
__device__ __forceinline__ void stage2(F2 (&v)[16], int ka, const F2* buf) {
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = buf[ka * kRS + i];
  Dft<float, 16>::run(v, SG, nullptr, 0);
}

// Z[j + 16 r] of a packed pair from the half spectra rows sa (line a) and sb (line b);
// DC and Nyquist take real parts; invalid lines read as zero.
__device__ __forceinline__ void load_half(F2 (&v)[16], const F2* sa, const F2* sb, int j, bool va, bool vb) {
  const F2 zero = cmake<float>(0.f, 0.f);
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int k = j + 16 * r;
    if (r < 8 || (r == 8 && j == 0)) {
      const F2 A = va ? sa[k] : zero, B = vb ? sb[k] : zero;
      v[r] = (k == 0 || k == 128) ? cmake<float>(A.x, B.x) : cmake<float>(A.x - B.y, A.y + B.x);
    } else {
      const int kk = 256 - k;
      const F2 A = va ? sa[kk] : zero, B = vb ? sb[kk] : zero;
      v[r] = cmake<float>(A.x + B.y, B.x - A.y);
    }
  }
}

// half spectra of the pair from its natural-order Z (thread j takes k = j + 16 r <= 128)
__device__ __forceinline__ void store_half(const F2* nat, F2* da, F2* db, int j, bool va, bool vb) {
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const int k = j + 16 * r;
    if (k > 128) break;
    const F2 Z = nat[k], W = nat[(256 - k) & 255];
    if (va) da[k] = cmake<float>((Z.x + W.x) * 0.5f, (Z.y - W.y) * 0.5f);
    if (vb) db[k] = cmake<float>((Z.y + W.y) * 0.5f, (W.x - Z.x) * 0.5f);
  }
}

// twiddle table by stage-1 output k (row) and thread j (column): entry 16 k + j holds
// W256^(j k), so the 16 threads of a pair read 16 consecutive entries (no bank conflicts)
__device__ __forceinline__ void init_tw(F2* tw) {
  for (int m = threadIdx.x; m < 256; m += blockDim.x) {
    float s, c;
    sincospif((float)((m >> 4) * (m & 15)) * (1.0f / 128.0f), &s, &c);
    tw[m] = cmake<float>(c, -s);
  }
}

}  // namespace x256

// Shared memory of the register x passes: twiddles, one transposition buffer per pair,
// and for the middle pass the six strains of each voxel.
// The middle pass stages the phase ids of its voxels (LX x 256 uint16) behind them; the
// operator epilogue stages p, the density source and the mask (xinv_stage_layout).
__host__ __device__ __forceinline__ constexpr size_t xreg_smem_mid(int lx) {
  return (size_t)(256 + 3 * lx * x256::kPairBuf + lx * 768) * sizeof(float2) + (size_t)lx * 256 * 2;
}
__host__ __device__ __forceinline__ constexpr size_t xreg_smem(int npairs) {
  return (size_t)(256 + npairs * x256::kPairBuf) * sizeof(float2);
}

// x middle pass: LX lines x 6 strain components = 3 LX pairs, 48 LX threads.
template <int BATCH>
__global__ void __launch_bounds__(256, 3) k_xmid256(const Desc<float>* __restrict__ dd, BatchArgs<float> ba) {
  using namespace x256;
  int blk;
  const Desc<float>* __restrict__ Dp = pick_ptr<float, BATCH>(dd, ba, blk);
  const Desc<float>& D = *Dp;
  if (D.sc->done) return;
  const int LX = D.lxm;
  extern __shared__ __align__(16) unsigned char smraw[];
  F2* tw = reinterpret_cast<F2*>(smraw);
  F2* S = tw + 256;
  F2* E = S + 3 * LX * kPairBuf;  // per line: (x, pair m) -> strains (2m, 2m + 1)
  uint16_t* sph = reinterpret_cast<uint16_t*>(E + LX * 768);
  const int t = threadIdx.x, j = t & 15, pr = t >> 4;
  const int l = pr / 3, m = pr - 3 * l;
  const long long nsp = (long long)D.n2 * D.n3;
  const long long l0 = (long long)blk * LX;
  // phase ids of the block's voxels: one contiguous run, copied while the FFTs run
  if (D.phase) {
    const long long nv = nsp - l0 < LX ? nsp - l0 : LX;
    stage_copy(sph, D.phase + l0 * 256, (size_t)nv * 256 * 2);
    stage_commit();
  }
  init_tw(tw);
  const long long line = l0 + l;
  const bool valid = line < nsp;
  F2* sa = D.spec + (long long)(2 * m) * D.Vh + line * D.pitch;
  F2* sb = sa + D.Vh;
  F2* buf = S + pr * kPairBuf;
  F2 v[16];
  load_half(v, sa, sb, j, valid, valid);
  __syncthreads();
  stage1<+1>(v, j, tw, buf);
  __syncthreads();
  stage2<+1>(v, j, buf);
  F2* El = E + l * 768;
#pragma unroll
  for (int kb = 0; kb < 16; ++kb) El[(j + 16 * kb) * 3 + m] = v[kb];
  if (D.phase) stage_wait();
  __syncthreads();
  // sigma = C(x) : e over the block's voxels (consecutive x across a warp)
  for (int e = t; e < LX * 256; e += blockDim.x) {
    const int ll = e >> 8, x = e & 255;
    const long long ln = l0 + ll;
    if (ln >= nsp) continue;
    const long long vox = ln * 256 + x;
    const long long row = D.phase ? (long long)sph[e] : vox;
    float C[24];
    load_row<float>(D.ctab + row * kCtabStride3, C, 24);
    F2* ev = E + ll * 768 + x * 3;
    const F2 e01 = ev[0], e23 = ev[1], e45 = ev[2];
    float ee[6] = {e01.x, e01.y, e23.x, e23.y, e45.x, e45.y};
    hooke3<float>(C, ee);
    ev[0] = cmake<float>(ee[0], ee[1]);
    ev[1] = cmake<float>(ee[2], ee[3]);
    ev[2] = cmake<float>(ee[4], ee[5]);
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = El[(j + 16 * r) * 3 + m];
  stage1<-1>(v, j, tw, buf);
  __syncthreads();
  stage2<-1>(v, j, buf);
  // natural order of Z in the strain area (every read of it preceded the barrier above)
  F2* nat = El + m * 256;
#pragma unroll
  for (int kb = 0; kb < 16; ++kb) nat[j + 16 * kb] = v[kb];
  __syncthreads();
  store_half(nat, sa, sb, j, valid, valid);
}

// Lines and components of pair pr of an x pass over nc = 3 components: real lines
// q = 2 pr, 2 pr + 1 of the (line, component) order q = line * 3 + component.
struct XPair {
  long long la, lb;  // global line indices
  int ka, kb;        // components
  bool va, vb;
};
__device__ __forceinline__ XPair xpair(int pr, long long l0, long long nsp) {
  XPair P;
  const int qa = 2 * pr, qb = qa + 1;
  P.la = l0 + qa / 3;
  P.lb = l0 + qb / 3;
  P.ka = qa % 3;
  P.kb = qb % 3;
  P.va = P.la < nsp;
  P.vb = P.lb < nsp;
  return P;
}

// x inverse pass, 3 LX / 2 pairs, 24 LX threads.
// POST_APPLY with stage != 0: p (3 components), the density source (phase ids or
// per-voxel densities) and the mask of the block's lines are copied to shared memory at
// the start (16-byte cp.async, one contiguous run each; the host stages only when the
// operand is 16-byte aligned), so they arrive while the spectra load and transform.
template <int POST, int BATCH>
__global__ void __launch_bounds__(256, POST == POST_APPLY ? 3 : 4) k_xinv256(const Desc<float>* __restrict__ dd, BatchArgs<float> ba,
                                                    int in_slot, int out_slot, int masked, int want_dot,
                                                    int stage) {
  using namespace x256;
  int blk;
  const Desc<float>* __restrict__ Dp = pick_ptr<float, BATCH>(dd, ba, blk);
  const Desc<float>& D = *Dp;
  Scalars* sc = D.sc;
  if (sc->done) return;
  const int LX = D.lx;
  extern __shared__ __align__(16) unsigned char smraw[];
  F2* tw = reinterpret_cast<F2*>(smraw);
  F2* S = tw + 256;
  const int t = threadIdx.x, j = t & 15, pr = t >> 4;
  init_tw(tw);
  const long long nsp = (long long)D.n2 * D.n3;
  const long long l0 = (long long)blk * LX;
  const XPair P = xpair(pr, l0, nsp);
  F2* sa = D.spec + (long long)P.ka * D.Vh + P.la * D.pitch;
  F2* sb = D.spec + (long long)P.kb * D.Vh + P.lb * D.pitch;
  F2* buf = S + pr * kPairBuf;
  const bool pfirst = POST == POST_PREC_PUPD && sc->first != 0;
  const float pbeta = POST == POST_PREC_PUPD ? (float)sc->beta : 0.f;
  unsigned char* stg = reinterpret_cast<unsigned char*>(S + (3 * LX / 2) * kPairBuf);
  const XStage SL = xinv_stage_layout(POST_APPLY, 3, LX, 256, D.phase != nullptr);
  const bool stg_on = POST == POST_APPLY && stage;
  if (stg_on) {
    const long long nv = nsp - l0 < LX ? nsp - l0 : LX;
    const size_t e = (size_t)nv * 256;
    for (int k = 0; k < 3; ++k)
      stage_copy(stg + SL.p + (size_t)k * LX * 256 * 4,
                 reinterpret_cast<const float*>(D.slot[in_slot]) + (long long)k * D.V + l0 * 256, e * 4);
    if (D.phase)
      stage_copy(stg + SL.rho, D.phase + l0 * 256, e * 2);
    else
      stage_copy(stg + SL.rho, D.rhotab + l0 * 256, e * 4);
    if (masked) stage_copy(stg + SL.mask, D.mask + l0 * 256, e);
    stage_commit();
  }
  F2 v[16];
  load_half(v, sa, sb, j, P.va, P.vb);
  __syncthreads();
  stage1<+1>(v, j, tw, buf);
  __syncthreads();
  stage2<+1>(v, j, buf);
  // real values of lines a (v.x) and b (v.y) at x = j + 16 kb
  const long long V = D.V;
  const long long va0 = P.la * 256 + j, vb0 = P.lb * 256 + j;  // voxel of kb = 0
  const long long ga = (long long)P.ka * V + va0, gb = (long long)P.kb * V + vb0;
  DotAcc<float> acc;
  if (POST == POST_APPLY) {
    const float* pin = reinterpret_cast<const float*>(D.slot[in_slot]);
    float* qout = reinterpret_cast<float*>(D.slot[out_slot]);
    if (stg_on) {
      stage_wait();
      __syncthreads();
    }
    // staged element of line l (block-local), x
    const int la = (int)(P.la - l0), lb = (int)(P.lb - l0);
    const float* sp = reinterpret_cast<const float*>(stg + SL.p);
    auto operand = [&](int k, int ll, long long g, int x) {
      return stg_on ? sp[(size_t)k * LX * 256 + ll * 256 + x] : pin[g];
    };
    auto density = [&](int ll, long long vox, int x) {
      if (!stg_on) return rho_at<float>(D, vox);
      const int e = ll * 256 + x;
      return D.phase ? D.rhotab[reinterpret_cast<const uint16_t*>(stg + SL.rho)[e]]
                     : reinterpret_cast<const float*>(stg + SL.rho)[e];
    };
    auto maskbyte = [&](int ll, long long vox, int x) {
      return stg_on ? stg[SL.mask + ll * 256 + x] : D.mask[vox];
    };
#pragma unroll
    for (int kb = 0; kb < 16; ++kb) {
      const int o = 16 * kb, x = j + o;
      if (P.va) {
        const float pv = operand(P.ka, la, ga + o, x);
        float q = v[kb].x + density(la, va0 + o, x) * pv;
        if (masked && ((maskbyte(la, va0 + o, x) >> P.ka) & 1)) q = 0.f;
        qout[ga + o] = q;
        acc.add_prod(pv, q);
      }
      if (P.vb) {
        const float pv = operand(P.kb, lb, gb + o, x);
        float q = v[kb].y + density(lb, vb0 + o, x) * pv;
        if (masked && ((maskbyte(lb, vb0 + o, x) >> P.kb) & 1)) q = 0.f;
        qout[gb + o] = q;
        acc.add_prod(pv, q);
      }
    }
    if (want_dot) {
      const double s = block_sum(acc.value());
      if (t == 0) D.part[PT_A][blk] = s;
    }
  } else {  // POST_PREC_PUPD
    float* p = reinterpret_cast<float*>(D.slot[SL_P]);
#pragma unroll
    for (int kb = 0; kb < 16; ++kb) {
      const int o = 16 * kb;
      float za = v[kb].x, zb = v[kb].y;
      if (masked && P.va && ((D.mask[va0 + o] >> P.ka) & 1)) za = 0.f;
      if (masked && P.vb && ((D.mask[vb0 + o] >> P.kb) & 1)) zb = 0.f;
      if (!pfirst) {
        if (P.va) za += pbeta * p[ga + o];
        if (P.vb) zb += pbeta * p[gb + o];
      }
      if (P.va) p[ga + o] = za;
      if (P.vb) p[gb + o] = zb;
      v[kb] = cmake<float>(P.va ? za : 0.f, P.vb ? zb : 0.f);
    }
    // forward transform of p from the same positions (x = j + 16 r)
    __syncthreads();  // every stage-2 read of the buffer is done
    stage1<-1>(v, j, tw, buf);
    __syncthreads();
    stage2<-1>(v, j, buf);
    __syncthreads();
#pragma unroll
    for (int kb = 0; kb < 16; ++kb) buf[j + 16 * kb] = v[kb];
    __syncthreads();
    store_half(buf, sa, sb, j, P.va, P.vb);
  }
}

// x forward pass with the search-direction residual update (PRE_RUPD, FP32 inner solve).
template <int BATCH>
__global__ void __launch_bounds__(256, 4) k_xfwd256_rupd(const Desc<float>* __restrict__ dd, BatchArgs<float> ba) {
  using namespace x256;
  int blk;
  const Desc<float>* __restrict__ Dp = pick_ptr<float, BATCH>(dd, ba, blk);
  const Desc<float>& D = *Dp;
  Scalars* sc = D.sc;
  if (sc->done) return;
  const int LX = D.lx;
  extern __shared__ __align__(16) unsigned char smraw[];
  F2* tw = reinterpret_cast<F2*>(smraw);
  F2* S = tw + 256;
  const int t = threadIdx.x, j = t & 15, pr = t >> 4;
  init_tw(tw);
  const long long nsp = (long long)D.n2 * D.n3;
  const long long l0 = (long long)blk * LX;
  const XPair P = xpair(pr, l0, nsp);
  const float alpha = (float)sc->alpha;
  const long long V = D.V;
  const long long ga = (long long)P.ka * V + P.la * 256 + j, gb = (long long)P.kb * V + P.lb * 256 + j;
  // the four vectors are distinct arrays (restrict): each chunk's loads of all four are
  // issued before its stores, kChunk points of both lines at a time
  const float* __restrict__ pp = reinterpret_cast<const float*>(D.slot[SL_P]);
  const float* __restrict__ qq = reinterpret_cast<const float*>(D.slot[SL_Q]);
  float* __restrict__ rr = reinterpret_cast<float*>(D.slot[SL_R]);
  float* __restrict__ dd32 = reinterpret_cast<float*>(D.slot[SL_D]);
  constexpr int kChunk = 2;
  DotAcc<float> acc;
  F2 v[16];
#pragma unroll
  for (int r0 = 0; r0 < 16; r0 += kChunk) {
    float pa[kChunk], qa[kChunk], ra_[kChunk], da[kChunk], pb[kChunk], qb[kChunk], rb_[kChunk], db[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int o = 16 * (r0 + u);
      pa[u] = P.va ? pp[ga + o] : 0.f;
      qa[u] = P.va ? qq[ga + o] : 0.f;
      ra_[u] = P.va ? rr[ga + o] : 0.f;
      da[u] = P.va ? dd32[ga + o] : 0.f;
      pb[u] = P.vb ? pp[gb + o] : 0.f;
      qb[u] = P.vb ? qq[gb + o] : 0.f;
      rb_[u] = P.vb ? rr[gb + o] : 0.f;
      db[u] = P.vb ? dd32[gb + o] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int o = 16 * (r0 + u);
      const float ra = ra_[u] - alpha * qa[u], rb = rb_[u] - alpha * qb[u];
      if (P.va) {
        dd32[ga + o] = da[u] + alpha * pa[u];
        rr[ga + o] = ra;
        acc.add_prod(ra, ra);
      }
      if (P.vb) {
        dd32[gb + o] = db[u] + alpha * pb[u];
        rr[gb + o] = rb;
        acc.add_prod(rb, rb);
      }
      v[r0 + u] = cmake<float>(ra, rb);
    }
  }
  {
    const double s = block_sum(acc.value());  // contains barriers (the twiddles are ready)
    if (t == 0) D.part[PT_A][blk] = s;
  }
  F2* buf = S + pr * kPairBuf;
  stage1<-1>(v, j, tw, buf);
  __syncthreads();
  stage2<-1>(v, j, buf);
  __syncthreads();
#pragma unroll
  for (int kb = 0; kb < 16; ++kb) buf[j + 16 * kb] = v[kb];
  __syncthreads();
  F2* sa = D.spec + (long long)P.ka * D.Vh + P.la * D.pitch;
  F2* sb = D.spec + (long long)P.kb * D.Vh + P.lb * D.pitch;
  store_half(buf, sa, sb, j, P.va, P.vb);
}

}  // namespace wfft
