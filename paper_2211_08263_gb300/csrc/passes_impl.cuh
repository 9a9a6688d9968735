// Launch sequences of the fused passes, instantiated per arithmetic type.
#pragma once
#include <algorithm>
#include <cmath>

#include "launch.cuh"
#include "passes.cuh"
#include "profiler.cuh"

namespace wfft {

// Largest tile (complex elements per block) whose every radix stage fits the
// per-thread register batch NbOf<T, R> with `thr` threads.
template <typename T>
static int max_tile_elems(const AxisPlan& pl, int thr) {
  int cap = 1 << 30;
  const int rad[6] = {8, 4, 2, 3, 5, 7};
  for (int i = 0; i < 6; ++i) {
    if (!pl.cnt[i]) continue;
    const int R = rad[i];
    const int capR = sizeof(T) == 8 ? 8 : 16;
    const int nb = std::max(1, capR / R);
    cap = std::min(cap, nb * R * thr);
  }
  return cap;
}

template <typename T>
void plan_geometry(Plan<T>& P) {
  const Desc<T>& D = P.h;
  PassGeo& g = P.g;
  g.thr = 256;
  const int budget = 2048;  // target complex elements per block tile
  const long long nsp = (long long)D.n2 * D.n3;
  // x passes: npairs * N1 <= elems, LX * nc even
  const int ex = std::min(budget, max_tile_elems<T>(D.ax[0], g.thr));
  auto pick_lx = [&](int nc) {
    int lx = std::max(1, (2 * ex) / (nc * D.n1));
    if (lx > nsp) lx = (int)std::max<long long>(1, nsp);
    while (lx > 1 && ((lx * nc) & 1)) --lx;
    if ((lx * nc) & 1) lx = 2;  // odd nc with a single line: pair two lines
    return lx;
  };
  g.LX = pick_lx(D.c);
  g.LXm = pick_lx(D.s);
  g.blk_x = (int)((nsp + g.LX - 1) / g.LX);
  g.blk_xm = (int)((nsp + g.LXm - 1) / g.LXm);
  const size_t cs = sizeof(cplx<T>);
  g.sm_x = (size_t)(D.n1 + (g.LX * D.c / 2) * D.n1) * cs;
  g.sm_xm = (size_t)(D.n1 + (g.LXm * D.s / 2) * D.n1) * cs;
  // column passes: per axis and op, the widest tile (kx columns) whose every
  // radix stage fits the register batch and whose slots fit 64 KB of shared memory
  const int maxbx = sizeof(T) == 4 ? 8 : 4;
  g.max_blocks = std::max(std::max(g.blk_x, g.blk_xm), 1);
  for (int ax = 0; ax < 3; ++ax)
    for (int op = 0; op < 5; ++op) {
      g.bx[ax][op] = 0;
      g.blk_col[ax][op] = 0;
      g.sm_col[ax][op] = 0;
    }
  for (int ax = 1; ax <= 2; ++ax) {
    const int N = ax == 1 ? D.n2 : D.n3;
    const int nouter = ax == 1 ? D.n3 : D.n2;
    for (int op = 0; op < 5; ++op) {
      const bool plain = op == OP_FWD || op == OP_INV;
      const int ns = plain ? 1 : (op == OP_PREC ? D.c : D.s);
      const int thr = plain ? kColThreadsPlain : kColThreadsOp;
      const int maxe = max_tile_elems<T>(D.ax[ax], thr);
      int bx = plain ? maxbx : std::min(maxbx, 4);
      while (bx > 1 && ((long long)ns * bx * N > maxe || (size_t)ns * bx * N * cs > 64 * 1024)) bx >>= 1;
      g.bx[ax][op] = bx;
      g.blk_col[ax][op] = ((D.nh + bx - 1) / bx) * nouter;
      g.sm_col[ax][op] = (size_t)(N + ns * bx * N) * cs;
      g.max_blocks = std::max(g.max_blocks, g.blk_col[ax][op]);
    }
  }
}

// ---------------------------------------------------------------------------
// algorithmic cost model of one launch (compulsory DRAM bytes: every input read
// once and every output written once, spectra at their unpadded size; flops:
// 5 N log2 N per complex FFT line, half that per real line, plus the pointwise work)
// ---------------------------------------------------------------------------
template <typename T>
struct Cost {
  double V, Vh, st, lg1, lg2, lg3, c, s;
  explicit Cost(const Desc<T>& D) {
    V = (double)D.V;
    Vh = (double)D.n3 * D.n2 * D.nh;
    st = sizeof(T);
    lg1 = std::log2((double)D.n1);
    lg2 = std::log2((double)D.n2);
    lg3 = std::log2((double)D.n3);
    c = D.c;
    s = D.s;
  }
  double spec(double ncomp) const { return ncomp * Vh * 2 * st; }
  double real(double ncomp) const { return ncomp * V * st; }
  double xfft(double ncomp) const { return 2.5 * V * lg1 * ncomp; }
  double colfft(int axis, double ncomp) const { return 5.0 * Vh * (axis == 1 ? lg2 : lg3) * ncomp; }
};
static inline int prec_index(size_t st) { return st == 8 ? 0 : 1; }

template <typename T>
static void launch_xfwd(const Plan<T>& P, int pre, int in_slot, cudaStream_t st) {
  const PassGeo& g = P.g;
  const Cost<T> k(P.h);
  const int pi = prec_index(sizeof(T));
  const double out = k.spec(k.c), fl = k.xfft(k.c);
  switch (pre) {
    case PRE_PLAIN:
      prof_launch(pi, KK_XFWD_PLAIN, k.real(k.c) + out, fl, st,
                  [&] { k_xfwd<T, PRE_PLAIN><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); });
      break;
    case PRE_PUPD:
      prof_launch(pi, KK_XFWD_PUPD, 3 * k.real(k.c) + out, fl + 2 * k.c * k.V, st,
                  [&] { k_xfwd<T, PRE_PUPD><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); });
      break;
    case PRE_RUPD:
      prof_launch(pi, KK_XFWD_RUPD, 6 * k.real(k.c) + out, fl + 6 * k.c * k.V, st,
                  [&] { k_xfwd<T, PRE_RUPD><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); });
      break;
    case PRE_CONV:
      prof_launch(pi, KK_XFWD_CONV, 8 * k.c * k.V + 2 * k.real(k.c) + out, fl + k.c * k.V, st,
                  [&] { k_xfwd<T, PRE_CONV><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); });
      break;
    default:  // PRE_XUPD: x += xcoef d (FP64 x, FP32 d), then transform x
      prof_launch(pi, KK_XFWD_PLAIN, 2 * k.real(k.c) + 4 * k.c * k.V + out, fl + 2 * k.c * k.V, st,
                  [&] { k_xfwd<T, PRE_XUPD><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); });
      break;
  }
}

template <typename T, int BX>
static void launch_colplain_bx(const Plan<T>& P, int op, int axis, int ncomp, cudaStream_t st) {
  const PassGeo& g = P.g;
  const dim3 grid(g.blk_col[axis][op], ncomp);
  const size_t sm = g.sm_col[axis][op];
  const Cost<T> k(P.h);
  const double by = 2 * k.spec(ncomp), fl = k.colfft(axis, ncomp);
  const int pi = prec_index(sizeof(T));
  if (op == OP_FWD)
    prof_launch(pi, KK_COL_FWD, by, fl, st,
                [&] { k_colplain<T, OP_FWD, BX><<<grid, kColThreadsPlain, sm, st>>>(P.d, axis); });
  else
    prof_launch(pi, KK_COL_INV, by, fl, st,
                [&] { k_colplain<T, OP_INV, BX><<<grid, kColThreadsPlain, sm, st>>>(P.d, axis); });
}

template <typename T, int OP, int BX>
static void launch_colop_bx(const Plan<T>& P, int axis, cudaStream_t st) {
  const PassGeo& g = P.g;
  const int nb = g.blk_col[axis][OP];
  const size_t sm = g.sm_col[axis][OP];
  const Cost<T> k(P.h);
  const bool d3 = P.h.ndim == 3;
  double by, fl;
  int kind;
  if (OP == OP_GRAD) {
    kind = KK_COL_GRAD;
    by = k.spec(k.c) + k.spec(k.s);
    fl = k.colfft(axis, k.c + k.s) + (d3 ? 42.0 : 20.0) * k.Vh;
  } else if (OP == OP_DIV) {
    kind = KK_COL_DIV;
    by = k.spec(k.s) + k.spec(k.c);
    fl = k.colfft(axis, k.c + k.s) + (d3 ? 36.0 : 16.0) * k.Vh;
  } else {
    kind = KK_COL_PREC;
    by = 2 * k.spec(k.c);
    fl = k.colfft(axis, 2 * k.c) + (d3 ? 100.0 : 40.0) * k.Vh;
  }
  // slots: c (2 or 3) for the preconditioner, s (3 or 6) for gradient / divergence
  constexpr int kSmall = OP == OP_PREC ? 2 : 3;
  constexpr int kLarge = OP == OP_PREC ? 3 : 6;
  prof_launch(prec_index(sizeof(T)), kind, by, fl, st, [&] {
    if (!d3)
      k_colop<T, OP, BX, kSmall><<<nb, kColThreadsOp, sm, st>>>(P.d, axis);
    else
      k_colop<T, OP, BX, kLarge><<<nb, kColThreadsOp, sm, st>>>(P.d, axis);
  });
}

template <typename T, int OP>
static void launch_colop(const Plan<T>& P, int axis, cudaStream_t st) {
  switch (P.g.bx[axis][OP]) {
    case 4: launch_colop_bx<T, OP, 4>(P, axis, st); break;
    case 2: launch_colop_bx<T, OP, 2>(P, axis, st); break;
    default: launch_colop_bx<T, OP, 1>(P, axis, st); break;
  }
}

template <typename T>
static void launch_col(const Plan<T>& P, int op, int axis, int ncomp, cudaStream_t st) {
  if (op == OP_FWD || op == OP_INV) {
    switch (P.g.bx[axis][op]) {
      case 8: launch_colplain_bx<T, 8>(P, op, axis, ncomp, st); break;
      case 4: launch_colplain_bx<T, 4>(P, op, axis, ncomp, st); break;
      case 2: launch_colplain_bx<T, 2>(P, op, axis, ncomp, st); break;
      default: launch_colplain_bx<T, 1>(P, op, axis, ncomp, st); break;
    }
    return;
  }
  if (op == OP_GRAD) launch_colop<T, OP_GRAD>(P, axis, st);
  else if (op == OP_DIV) launch_colop<T, OP_DIV>(P, axis, st);
  else launch_colop<T, OP_PREC>(P, axis, st);
}

template <typename T>
static void launch_xinv(const Plan<T>& P, int post, int in_slot, int out_slot, int masked, int want_dot,
                        cudaStream_t st) {
  const PassGeo& g = P.g;
  const Cost<T> k(P.h);
  const int pi = prec_index(sizeof(T));
  const double in = k.spec(k.c), fl = k.xfft(k.c);
  const double mat = (P.h.phase ? 2.0 : 0.0) * k.V + k.V;  // phase ids + mask bytes
  switch (post) {
    case POST_APPLY:
      prof_launch(pi, KK_XINV_APPLY, in + 2 * k.real(k.c) + mat, fl + 2 * k.c * k.V, st, [&] {
        k_xinv<T, POST_APPLY><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot, out_slot, masked, want_dot);
      });
      break;
    case POST_RESID:
      prof_launch(pi, KK_XINV_RESID, in + 24 * k.c * k.V + mat, fl + 3 * k.c * k.V, st, [&] {
        k_xinv<T, POST_RESID><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot, out_slot, masked, want_dot);
      });
      break;
    default:
      prof_launch(pi, KK_XINV_PREC, in + k.real(k.c) + k.V, fl, st, [&] {
        k_xinv<T, POST_PREC><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot, out_slot, masked, 0);
      });
      break;
  }
}

template <typename T>
void launch_apply(const Plan<T>& P, int pre, int in_slot, int post, int out_slot, int masked, int want_dot,
                  cudaStream_t st) {
  const Desc<T>& D = P.h;
  launch_xfwd<T>(P, pre, in_slot, st);
  if (D.midAxis) launch_col<T>(P, OP_FWD, D.midAxis, D.c, st);
  launch_col<T>(P, OP_GRAD, D.opAxis, D.c, st);
  if (D.midAxis) launch_col<T>(P, OP_INV, D.midAxis, D.s, st);
  {
    const Cost<T> k(D);
    const double by = 2 * k.spec(k.s) + (D.phase ? 2.0 : 0.0) * k.V;
    const double fl = 2 * k.xfft(k.s) + (D.ndim == 3 ? 66.0 : 15.0) * k.V;
    prof_launch(prec_index(sizeof(T)), KK_XMID, by, fl, st,
                [&] { k_xmid<T><<<P.g.blk_xm, P.g.thr, P.g.sm_xm, st>>>(P.d, P.g.LXm); });
  }
  if (D.midAxis) launch_col<T>(P, OP_FWD, D.midAxis, D.s, st);
  launch_col<T>(P, OP_DIV, D.opAxis, D.c, st);
  if (D.midAxis) launch_col<T>(P, OP_INV, D.midAxis, D.c, st);
  // PRE_PUPD writes p; the epilogue reads the operator's input from in_slot
  launch_xinv<T>(P, post, pre == PRE_PUPD ? (int)SL_P : in_slot, out_slot, masked, want_dot, st);
}

template <typename T>
void launch_precond(const Plan<T>& P, int pre, int in_slot, int out_slot, int masked, cudaStream_t st) {
  const Desc<T>& D = P.h;
  launch_xfwd<T>(P, pre, in_slot, st);
  if (D.midAxis) launch_col<T>(P, OP_FWD, D.midAxis, D.c, st);
  launch_col<T>(P, OP_PREC, D.opAxis, D.c, st);
  if (D.midAxis) launch_col<T>(P, OP_INV, D.midAxis, D.c, st);
  launch_xinv<T>(P, POST_PREC, in_slot, out_slot, masked, 0, st);
}

// Plain 3-D transforms for testing: the x pass with c replaced by ncomp.
template <typename T>
__global__ void __launch_bounds__(256) k_xplain(const Desc<T>* __restrict__ dd, int LX, int nc, int dir, int slot) {
  const Desc<T>& D = *dd;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = D.n1;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* buf = tw + N;
  const long long nsp = (long long)D.n2 * D.n3;
  const long long l0 = (long long)blockIdx.x * LX;
  load_twiddles<T>(tw, D.tw[0], N);
  T* f = reinterpret_cast<T*>(D.slot[slot]);
  if (dir < 0) {
    for (int e = threadIdx.x; e < LX * nc * N; e += blockDim.x) {
      const int x = e % N, q = e / N, k = q % nc, l = q / nc;
      const long long line = l0 + l;
      packed<T>(buf, N, q, x) = line < nsp ? f[(long long)k * D.V + line * N + x] : (T)0;
    }
    __syncthreads();
    fft_lines<T, 1>(buf, D.ax[0], LX * nc / 2, N, tw, -1);
    store_unpacked<T>(D, buf, N, LX * nc, l0, nc, nsp);
  } else {
    load_packed<T>(D, buf, N, LX * nc, l0, nc, nsp);
    __syncthreads();
    fft_lines<T, 1>(buf, D.ax[0], LX * nc / 2, N, tw, +1);
    for (int e = threadIdx.x; e < LX * nc * N; e += blockDim.x) {
      const int x = e % N, q = e / N, k = q % nc, l = q / nc;
      const long long line = l0 + l;
      if (line < nsp) f[(long long)k * D.V + line * N + x] = packed<T>(buf, N, q, x);
    }
  }
}

template <typename T>
void launch_rfft3(const Plan<T>& P, int dir, int ncomp, int real_slot, cudaStream_t st) {
  const Desc<T>& D = P.h;
  const PassGeo& g = P.g;
  const long long nsp = (long long)D.n2 * D.n3;
  const int ex = std::min(2048, max_tile_elems<T>(D.ax[0], g.thr));
  int lx = std::max(1, (2 * ex) / (ncomp * D.n1));
  if (lx > nsp) lx = (int)std::max<long long>(1, nsp);
  while (lx > 1 && ((lx * ncomp) & 1)) --lx;
  if ((lx * ncomp) & 1) lx = 2;
  const int nb = (int)((nsp + lx - 1) / lx);
  const size_t sm = (size_t)(D.n1 + (lx * ncomp / 2) * D.n1) * sizeof(cplx<T>);
  const int axes[2] = {1, 2};
  if (dir < 0) {
    prof_launch(prec_index(sizeof(T)), KK_XFWD_PLAIN, Cost<T>(D).real(ncomp) + Cost<T>(D).spec(ncomp),
                Cost<T>(D).xfft(ncomp), st, [&] { k_xplain<T><<<nb, g.thr, sm, st>>>(P.d, lx, ncomp, -1, real_slot); });
    for (int a : axes)
      if ((a == 1 ? D.n2 : D.n3) > 1) launch_col<T>(P, OP_FWD, a, ncomp, st);
  } else {
    for (int a : {2, 1})
      if ((a == 1 ? D.n2 : D.n3) > 1) launch_col<T>(P, OP_INV, a, ncomp, st);
    prof_launch(prec_index(sizeof(T)), KK_XINV_PREC, Cost<T>(D).real(ncomp) + Cost<T>(D).spec(ncomp),
                Cost<T>(D).xfft(ncomp), st, [&] { k_xplain<T><<<nb, g.thr, sm, st>>>(P.d, lx, ncomp, +1, real_slot); });
  }
}

template <typename T>
cudaError_t init_kernel_attributes() {
  const int maxsm = 200 * 1024;  // opt-in limit minus the static shared memory of the reductions
  cudaError_t e = cudaSuccess;
#define WFFT_SETATTR(k)                                                                    \
  do {                                                                                     \
    cudaError_t ee = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm); \
    if (ee != cudaSuccess) e = ee;                                                         \
  } while (0)
  WFFT_SETATTR((k_xfwd<T, PRE_PLAIN>));
  WFFT_SETATTR((k_xfwd<T, PRE_PUPD>));
  WFFT_SETATTR((k_xfwd<T, PRE_RUPD>));
  WFFT_SETATTR((k_xfwd<T, PRE_CONV>));
  WFFT_SETATTR((k_xfwd<T, PRE_XUPD>));
  WFFT_SETATTR((k_xinv<T, POST_APPLY>));
  WFFT_SETATTR((k_xinv<T, POST_RESID>));
  WFFT_SETATTR((k_xinv<T, POST_PREC>));
  WFFT_SETATTR((k_xmid<T>));
  WFFT_SETATTR((k_xplain<T>));
#define WFFT_SETATTR_BX(BXV)                  \
  WFFT_SETATTR((k_colop<T, OP_GRAD, BXV, 3>));  \
  WFFT_SETATTR((k_colop<T, OP_GRAD, BXV, 6>));  \
  WFFT_SETATTR((k_colop<T, OP_DIV, BXV, 3>));   \
  WFFT_SETATTR((k_colop<T, OP_DIV, BXV, 6>));   \
  WFFT_SETATTR((k_colop<T, OP_PREC, BXV, 2>));  \
  WFFT_SETATTR((k_colop<T, OP_PREC, BXV, 3>));
  WFFT_SETATTR_BX(1)
  WFFT_SETATTR_BX(2)
  WFFT_SETATTR_BX(4)
  WFFT_SETATTR((k_colplain<T, OP_FWD, 1>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 1>));
  WFFT_SETATTR((k_colplain<T, OP_FWD, 2>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 2>));
  WFFT_SETATTR((k_colplain<T, OP_FWD, 4>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 4>));
  WFFT_SETATTR((k_colplain<T, OP_FWD, 8>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 8>));
#undef WFFT_SETATTR_BX
#undef WFFT_SETATTR
  return e;
}

#define WFFT_INSTANTIATE(T)                                                                                  \
  template void plan_geometry<T>(Plan<T>&);                                                                  \
  template void launch_apply<T>(const Plan<T>&, int, int, int, int, int, int, cudaStream_t);                \
  template void launch_precond<T>(const Plan<T>&, int, int, int, int, cudaStream_t);                        \
  template void launch_rfft3<T>(const Plan<T>&, int, int, int, cudaStream_t);                               \
  template cudaError_t init_kernel_attributes<T>();

}  // namespace wfft
