// Launch sequences of the fused passes, instantiated per arithmetic type.
#pragma once
#include <algorithm>

#include "launch.cuh"
#include "passes.cuh"

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
  // column passes: BX consecutive kx columns (64-byte rows) within the budget
  int bx = sizeof(T) == 4 ? 8 : 4;
  int ecol = budget;
  for (int ax = 1; ax <= 2; ++ax) ecol = std::min(ecol, max_tile_elems<T>(D.ax[ax], g.thr));
  const int nmax = std::max(D.n2, D.n3);
  while (bx > 1 && bx * nmax > ecol) bx >>= 1;
  g.BX = bx;
  const int ntx = (D.nh + bx - 1) / bx;
  g.blk_col[0] = 0;
  g.blk_col[1] = ntx * D.n3;
  g.blk_col[2] = ntx * D.n2;
  for (int ax = 1; ax <= 2; ++ax) {
    const int N = ax == 1 ? D.n2 : D.n3;
    const size_t tile = (size_t)bx * N * cs;
    g.sm_col[ax][OP_FWD] = N * cs + tile;
    g.sm_col[ax][OP_INV] = N * cs + tile;
    g.sm_col[ax][OP_GRAD] = N * cs + (D.c + 1) * tile;
    g.sm_col[ax][OP_DIV] = N * cs + (D.c + 1) * tile;
    g.sm_col[ax][OP_PREC] = N * cs + D.c * tile;
  }
  g.max_blocks = std::max(std::max(g.blk_x, g.blk_xm), std::max(std::max(g.blk_col[1], g.blk_col[2]), 1));
}

template <typename T>
static void launch_xfwd(const Plan<T>& P, int pre, int in_slot, cudaStream_t st) {
  const PassGeo& g = P.g;
  switch (pre) {
    case PRE_PLAIN: k_xfwd<T, PRE_PLAIN><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); break;
    case PRE_PUPD: k_xfwd<T, PRE_PUPD><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); break;
    case PRE_RUPD: k_xfwd<T, PRE_RUPD><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); break;
    default: k_xfwd<T, PRE_CONV><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot); break;
  }
}

template <typename T>
static void launch_col(const Plan<T>& P, int op, int axis, int ncomp, cudaStream_t st) {
  const PassGeo& g = P.g;
  const int nb = g.blk_col[axis];
  const size_t sm = g.sm_col[axis][op];
  switch (op) {
    case OP_FWD: k_col<T, OP_FWD><<<nb, g.thr, sm, st>>>(P.d, axis, g.BX, ncomp); break;
    case OP_INV: k_col<T, OP_INV><<<nb, g.thr, sm, st>>>(P.d, axis, g.BX, ncomp); break;
    case OP_GRAD: k_col<T, OP_GRAD><<<nb, g.thr, sm, st>>>(P.d, axis, g.BX, ncomp); break;
    case OP_DIV: k_col<T, OP_DIV><<<nb, g.thr, sm, st>>>(P.d, axis, g.BX, ncomp); break;
    default: k_col<T, OP_PREC><<<nb, g.thr, sm, st>>>(P.d, axis, g.BX, ncomp); break;
  }
}

template <typename T>
static void launch_xinv(const Plan<T>& P, int post, int in_slot, int out_slot, int masked, int want_dot,
                        cudaStream_t st) {
  const PassGeo& g = P.g;
  switch (post) {
    case POST_APPLY:
      k_xinv<T, POST_APPLY><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot, out_slot, masked, want_dot);
      break;
    case POST_RESID:
      k_xinv<T, POST_RESID><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot, out_slot, masked, want_dot);
      break;
    default:
      k_xinv<T, POST_PREC><<<g.blk_x, g.thr, g.sm_x, st>>>(P.d, g.LX, in_slot, out_slot, masked, 0);
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
  k_xmid<T><<<P.g.blk_xm, P.g.thr, P.g.sm_xm, st>>>(P.d, P.g.LXm);
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
    fft_lines<T>(buf, D.ax[0], LX * nc / 2, N, 1, tw, -1, false);
    store_unpacked<T>(D, buf, N, LX * nc, l0, nc, nsp);
  } else {
    load_packed<T>(D, buf, N, LX * nc, l0, nc, nsp);
    __syncthreads();
    fft_lines<T>(buf, D.ax[0], LX * nc / 2, N, 1, tw, +1, false);
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
    k_xplain<T><<<nb, g.thr, sm, st>>>(P.d, lx, ncomp, -1, real_slot);
    for (int a : axes)
      if ((a == 1 ? D.n2 : D.n3) > 1) launch_col<T>(P, OP_FWD, a, ncomp, st);
  } else {
    for (int a : {2, 1})
      if ((a == 1 ? D.n2 : D.n3) > 1) launch_col<T>(P, OP_INV, a, ncomp, st);
    k_xplain<T><<<nb, g.thr, sm, st>>>(P.d, lx, ncomp, +1, real_slot);
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
  WFFT_SETATTR((k_xinv<T, POST_APPLY>));
  WFFT_SETATTR((k_xinv<T, POST_RESID>));
  WFFT_SETATTR((k_xinv<T, POST_PREC>));
  WFFT_SETATTR((k_xmid<T>));
  WFFT_SETATTR((k_xplain<T>));
  WFFT_SETATTR((k_col<T, OP_FWD>));
  WFFT_SETATTR((k_col<T, OP_INV>));
  WFFT_SETATTR((k_col<T, OP_GRAD>));
  WFFT_SETATTR((k_col<T, OP_DIV>));
  WFFT_SETATTR((k_col<T, OP_PREC>));
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
