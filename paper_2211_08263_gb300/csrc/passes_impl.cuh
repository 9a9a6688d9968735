// Launch sequences of the fused passes, instantiated per arithmetic type.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cmath>

#include "launch.cuh"
#include "passes.cuh"
#include "col256.cuh"
#include "xreg256.cuh"
#include "profiler.cuh"

namespace wfft {

// Largest tile (complex elements per block) whose every radix stage fits the
// per-thread register batch NbOf<T, R> with `thr` threads.
template <typename T>
static int max_tile_elems(const AxisPlan& pl, int thr) {
  int cap = 1 << 30;
  // elements per thread of one stage, radix order 8, 4, 2, 3, 5, 7, 16 (the stage's own rule)
  const int per[7] = {8 * NbOf<T, 8>::v, 4 * NbOf<T, 4>::v, 2 * NbOf<T, 2>::v, 3 * NbOf<T, 3>::v,
                      5 * NbOf<T, 5>::v, 7 * NbOf<T, 7>::v, 16 * NbOf<T, 16>::v};
  for (int i = 0; i < 7; ++i)
    if (pl.cnt[i]) cap = std::min(cap, per[i] * thr);
  // the general prime stage: kPrimeBatch outputs per thread
  if (pl.prime) cap = std::min(cap, kPrimeBatch * thr);
  return cap;
}

// Dynamic shared memory a pass may request (the kernels' opt-in attribute).
constexpr size_t kMaxDynSmem = 200 * 1024;

// x lines per block of an x pass over nc components with at most `ex` complex
// elements per tile: lines are transformed in pairs (two real lines as one complex
// line), so lx * nc is even; a single line of an odd nc takes two lines (nc pairs).
static inline int x_tile_lines(int n1, long long nsp, int ex, int nc) {
  int lx = std::max(1, (2 * ex) / (nc * n1));
  if (lx > nsp) lx = (int)std::max<long long>(1, nsp);
  while (lx > 1 && ((lx * nc) & 1)) --lx;
  if ((lx * nc) & 1) lx = 2;
  return lx;
}

// Whether an x pass over nc components fits: its tile of lx * nc / 2 line pairs within
// the register batch of every stage, and its shared memory within the opt-in limit.
template <typename T>
static bool x_tile_fits(const Desc<T>& D, int thr, int lx, int nc) {
  const long long elems = (long long)(lx * nc / 2) * D.n1;
  const size_t sm = (size_t)(D.n1 + (lx * nc / 2) * row_stride(D.n1)) * sizeof(cplx<T>);
  return elems <= max_tile_elems<T>(D.ax[0], thr) && sm <= kMaxDynSmem;
}

// Slots transformed by one batched FFT call of a column pass: the 3-D gradient and
// divergence passes transform their six strain / stress slots as two batches of three.
static inline int col_batch_slots(int op, int ns) {
  return (op == OP_GRAD || op == OP_DIV) && ns == 6 ? 3 : ns;
}

template <typename T>
void plan_geometry(Plan<T>& P) {
  Desc<T>& D = P.h;
  PassGeo& g = P.g;
  g.thr = 256;
  const int xe = g.xelems & (kXReg - 1);
  const int budget = xe > 0 ? xe : 2048;  // target complex elements per x-pass tile
  const long long nsp = (long long)D.n2 * D.n3;
  // x passes: npairs * N1 <= elems, LX * nc even
  const int ex = std::min(budget, max_tile_elems<T>(D.ax[0], g.thr));
  g.LX = x_tile_lines(D.n1, nsp, ex, D.c);
  g.LXm = x_tile_lines(D.n1, nsp, ex, D.s);
  g.fits = x_tile_fits(D, g.thr, g.LX, D.c) && x_tile_fits(D, g.thr, g.LXm, D.s);
  P.h.lx = g.LX;
  P.h.lxm = g.LXm;
  g.blk_x = (int)((nsp + g.LX - 1) / g.LX);
  g.blk_xm = (int)((nsp + g.LXm - 1) / g.LXm);
  const size_t cs = sizeof(cplx<T>);
  g.sm_x = (size_t)(D.n1 + (g.LX * D.c / 2) * row_stride(D.n1)) * cs;
  g.sm_xm = (size_t)(D.n1 + (g.LXm * D.s / 2) * row_stride(D.n1)) * cs;
  // register-stage x passes: FP32 3-D grids with 256-point rows, at most 256 threads per
  // block (16 per line pair: 24 LX for the c-component passes, 48 LXm for the middle pass)
  g.xreg = false;
  if (g.xelems & kXReg) {
    const bool ok = sizeof(T) == 4 && D.ndim == 3 && D.c == 3 && D.s == 6 && D.n1 == 256 && g.LX % 2 == 0 &&
                    24 * g.LX <= 256 && 48 * g.LXm <= 256 && xreg_smem_mid(g.LXm) <= kMaxDynSmem;
    if (ok) g.xreg = true;
    else g.fits = false;
  }
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
      const int nb = col_batch_slots(op, ns);
      const int thr = plain ? kColThreadsPlain : kColThreadsOp;
      const int maxe = max_tile_elems<T>(D.ax[ax], thr);
      int bx = plain ? maxbx : std::min(maxbx, 4);
      while (bx > 1 && ((long long)nb * bx * N > maxe || (size_t)col_es(ns, bx, sizeof(T)) * N * cs > 64 * 1024))
        bx >>= 1;
      g.bx[ax][op] = bx;
      g.blk_col[ax][op] = ((D.nh + bx - 1) / bx) * nouter;
      g.sm_col[ax][op] = (size_t)(N + col_es(ns, bx, sizeof(T)) * N) * cs;
      g.max_blocks = std::max(g.max_blocks, g.blk_col[ax][op]);
      if (N > 1 && ((long long)nb * bx * N > maxe || g.sm_col[ax][op] > kMaxDynSmem)) g.fits = false;
    }
  }
}

// Column-tile width bx of pass (axis, op): feasible when every radix stage fits the
// per-thread register batch and the tile fits 64 KB of shared memory (the rule
// plan_geometry applies to its default choice); set_col_bx applies it to the plan.
// The register-stage kernels (k_col256) take FP32 3-D grids with a 256-point axis: plain
// transforms on any column axis, the fused passes on the axis hosting the spectral
// multiply.  They do not depend on the axis' radix schedule.
template <typename T>
static bool col256_ok(const Desc<T>& D, int axis, int op) {
  const int N = axis == 1 ? D.n2 : D.n3;
  if (sizeof(T) != 4 || D.ndim != 3 || D.c != 3 || D.s != 6 || N != 256) return false;
  return op == OP_FWD || op == OP_INV || axis == D.opAxis;
}

template <typename T>
bool col_bx_feasible(const Plan<T>& P, int axis, int op, int bx) {
  const Desc<T>& D = P.h;
  const int N = axis == 1 ? D.n2 : D.n3;
  const bool plain = op == OP_FWD || op == OP_INV;
  const int ns = plain ? 1 : (op == OP_PREC ? D.c : D.s);
  const int thr = plain ? kColThreadsPlain : kColThreadsOp;
  if (col_is_reg(bx)) {
    const int w = col_width(bx);
    return (w == 4 || w == 8 || w == 16) && bx == (kColReg | w) && col256_ok(D, axis, op);
  }
  const int maxbx = plain && sizeof(T) == 4 ? 16 : 4;  // 16-wide plain tiles: FP32 only (tuned, not default)
  if (bx < 1 || bx > maxbx || (bx & (bx - 1))) return false;
  const size_t sm = (size_t)(N + col_es(ns, bx, sizeof(T)) * N) * sizeof(cplx<T>);
  return (long long)col_batch_slots(op, ns) * bx * N <= max_tile_elems<T>(D.ax[axis], thr) &&
         ((size_t)col_es(ns, bx, sizeof(T)) * N * sizeof(cplx<T>) <= 64 * 1024 || (bx == 1 && sm <= kMaxDynSmem));
}

template <typename T>
void set_col_bx(Plan<T>& P, int axis, int op, int bx) {
  const Desc<T>& D = P.h;
  const int N = axis == 1 ? D.n2 : D.n3;
  const int nouter = axis == 1 ? D.n3 : D.n2;
  const bool plain = op == OP_FWD || op == OP_INV;
  const int ns = plain ? 1 : (op == OP_PREC ? D.c : D.s);
  const int w = col_width(bx);
  P.g.bx[axis][op] = bx;
  P.g.blk_col[axis][op] = ((D.nh + w - 1) / w) * nouter;
  P.g.sm_col[axis][op] = col_is_reg(bx) ? col256_smem(plain ? 1 : 3, w)
                                         : (size_t)(N + col_es(ns, bx, sizeof(T)) * N) * sizeof(cplx<T>);
  P.g.max_blocks = std::max(P.g.max_blocks, P.g.blk_col[axis][op]);
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
// profile slot of an arithmetic type: 0 FP64, 1 FP32
template <typename T> constexpr int prec_of() { return sizeof(T) == 8 ? 0 : 1; }

// ---------------------------------------------------------------------------
// launch helpers: one code path for single-instance and grouped launches
// ---------------------------------------------------------------------------
template <typename T>
int geo_blocks(const Plan<T>& P, int cls, int bx) {
  const Desc<T>& D = P.h;
  if (cls == GEO_X) return P.g.blk_x;
  if (cls == GEO_XM) return P.g.blk_xm;
  if (cls == GEO_EW) {
    const long long tot = (long long)D.c * D.V;
    return (int)std::min<long long>(std::max<long long>((tot + 255) / 256, 1), 1216);
  }
  const int axis = (cls - GEO_COL0) / 5 + 1;
  const int nouter = axis == 1 ? D.n3 : D.n2;
  const int w = col_width(bx);
  return ((D.nh + w - 1) / w) * nouter;
}

template <typename T>
size_t geo_smem(const Plan<T>& P, int cls, int bx) {
  const Desc<T>& D = P.h;
  const size_t cs = sizeof(cplx<T>);
  if (cls == GEO_X) return P.g.sm_x;
  if (cls == GEO_XM) return P.g.sm_xm;
  if (cls == GEO_EW) return 0;
  const int axis = (cls - GEO_COL0) / 5 + 1, op = (cls - GEO_COL0) % 5;
  const int N = axis == 1 ? D.n2 : D.n3;
  const bool plain = op == OP_FWD || op == OP_INV;
  const int ns = plain ? 1 : (op == OP_PREC ? D.c : D.s);
  if (col_is_reg(bx)) return col256_smem(plain ? 1 : 3, col_width(bx));
  return (size_t)(N + col_es(ns, bx, (int)sizeof(T)) * N) * cs;
}

template <typename T, int B>
struct Launch {
  const Plan<T>& P;
  const BatchLaunch<T>* bl;
  int grid(int cls) const {
    if (bl) return bl->total[cls];
    if (cls == GEO_X) return P.g.blk_x;
    if (cls == GEO_XM) return P.g.blk_xm;
    const int axis = (cls - GEO_COL0) / 5 + 1, op = (cls - GEO_COL0) % 5;
    return P.g.blk_col[axis][op];
  }
  size_t smem(int cls) const {
    if (bl) return bl->sm[cls];
    if (cls == GEO_X) return P.g.sm_x;
    if (cls == GEO_XM) return P.g.sm_xm;
    const int axis = (cls - GEO_COL0) / 5 + 1, op = (cls - GEO_COL0) % 5;
    return P.g.sm_col[axis][op];
  }
  int bx(int axis, int op) const { return bl ? bl->bx[axis][op] : P.g.bx[axis][op]; }
  BatchArgs<T> args(int cls) const {
    BatchArgs<T> a;
    a.descs = bl ? bl->descs : nullptr;
    a.start = bl ? bl->start[cls] : nullptr;
    a.n = bl ? bl->n : 0;
    return a;
  }
  // summed cost model over the instances of the launch
  template <typename F>
  void cost(F&& f, double& bytes, double& flops) const {
    bytes = flops = 0.0;
    if (!bl) {
      f(P, bytes, flops);
      return;
    }
    for (const Plan<T>* q : bl->plans) {
      double b = 0, fl = 0;
      f(*q, b, fl);
      bytes += b;
      flops += fl;
    }
  }
};

template <typename T, int B>
static void launch_xfwd(const Launch<T, B>& L, int pre, int in_slot, cudaStream_t st) {
  const int pi = prec_of<T>();
  const int nb = L.grid(GEO_X);
  const size_t sm = L.smem(GEO_X);
  const BatchArgs<T> ba = L.args(GEO_X);
  const Desc<T>* d = L.P.d;
  double by, fl;
  L.cost(
      [&](const Plan<T>& Q, double& b, double& f) {
        const Cost<T> k(Q.h);
        const double out = k.spec(k.c);
        f = k.xfft(k.c);
        switch (pre) {
          case PRE_PLAIN: b = k.real(k.c) + out; break;
          case PRE_PUPD: b = 3 * k.real(k.c) + out; f += 2 * k.c * k.V; break;
          case PRE_RUPD: b = 6 * k.real(k.c) + out; f += 6 * k.c * k.V; break;
          case PRE_CONV: b = 8 * k.c * k.V + 2 * k.real(k.c) + out; f += k.c * k.V; break;
          case PRE_CONVD: b = 8 * k.c * k.V + 4 * k.real(k.c) + out; f += 3 * k.c * k.V; break;
          default: b = 2 * k.real(k.c) + 4 * k.c * k.V + out; f += 2 * k.c * k.V; break;
        }
      },
      by, fl);
  switch (pre) {
    case PRE_PLAIN:
      prof_launch(pi, KK_XFWD_PLAIN, by, fl, st, [&] { k_xfwd<T, PRE_PLAIN, B><<<nb, 256, sm, st>>>(d, ba, in_slot); });
      break;
    case PRE_PUPD:
      prof_launch(pi, KK_XFWD_PUPD, by, fl, st, [&] { k_xfwd<T, PRE_PUPD, B><<<nb, 256, sm, st>>>(d, ba, in_slot); });
      break;
    case PRE_RUPD:
      if constexpr (B == 0 && sizeof(T) == 4) {
        if (L.P.g.xreg) {
          const int lx = L.P.h.lx;
          prof_launch(pi, KK_XFWD_RUPD, by, fl, st, [&] {
            k_xfwd256_rupd<B><<<nb, 24 * lx, xreg_smem(3 * lx / 2), st>>>(d, ba);
          });
          break;
        }
      }
      prof_launch(pi, KK_XFWD_RUPD, by, fl, st, [&] { k_xfwd<T, PRE_RUPD, B><<<nb, 256, sm, st>>>(d, ba, in_slot); });
      break;
    case PRE_CONV:
      prof_launch(pi, KK_XFWD_CONV, by, fl, st, [&] { k_xfwd<T, PRE_CONV, B><<<nb, 256, sm, st>>>(d, ba, in_slot); });
      break;
    case PRE_CONVD:
      if constexpr (B == 0 && sizeof(T) == 4)
        prof_launch(pi, KK_XFWD_CONV, by, fl, st, [&] { k_xfwd<T, PRE_CONVD, B><<<nb, 256, sm, st>>>(d, ba, in_slot); });
      break;
    default:  // PRE_XUPD: x += xcoef d (FP64 x, FP32 d), then transform x
      prof_launch(pi, KK_XFWD_PLAIN, by, fl, st, [&] { k_xfwd<T, PRE_XUPD, B><<<nb, 256, sm, st>>>(d, ba, in_slot); });
      break;
  }
}

template <typename T, int BX, int B>
static void launch_colplain_bx(const Launch<T, B>& L, int op, int axis, int ncomp, cudaStream_t st) {
  const int cls = geo_col(axis, op);
  const dim3 grid(L.grid(cls), ncomp);
  const size_t sm = L.smem(cls);
  const BatchArgs<T> ba = L.args(cls);
  const Desc<T>* d = L.P.d;
  double by, fl;
  L.cost(
      [&](const Plan<T>& Q, double& b, double& f) {
        const Cost<T> k(Q.h);
        b = 2 * k.spec(ncomp);
        f = k.colfft(axis, ncomp);
      },
      by, fl);
  const int pi = prec_of<T>();
  if (op == OP_FWD)
    prof_launch(pi, KK_COL_FWD, by, fl, st,
                [&] { k_colplain<T, OP_FWD, BX, B><<<grid, kColThreadsPlain, sm, st>>>(d, ba, axis); });
  else
    prof_launch(pi, KK_COL_INV, by, fl, st,
                [&] { k_colplain<T, OP_INV, BX, B><<<grid, kColThreadsPlain, sm, st>>>(d, ba, axis); });
}

// Register-stage pass over a 256-point axis (FP32): plain transforms of ncomp components
// (grid.y) or the fused gradient / divergence / preconditioner pass.
template <typename T, int OP, int BXC, int B>
static void launch_col256(const Launch<T, B>& L, int axis, int ncomp, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    const int cls = geo_col(axis, OP);
    const bool plain = OP == OP_FWD || OP == OP_INV;
    const dim3 grid(L.grid(cls), plain ? ncomp : 1);
    const size_t sm = L.smem(cls);
    const BatchArgs<T> ba = L.args(cls);
    const Desc<T>* d = L.P.d;
    double by, fl;
    L.cost(
        [&](const Plan<T>& Q, double& b, double& f) {
          const Cost<T> k(Q.h);
          if (OP == OP_FWD || OP == OP_INV) {
            b = 2 * k.spec(ncomp);
            f = k.colfft(axis, ncomp);
          } else if (OP == OP_GRAD) {
            b = k.spec(k.c) + k.spec(k.s);
            f = k.colfft(axis, k.c + k.s) + 42.0 * k.Vh;
          } else if (OP == OP_DIV) {
            b = k.spec(k.s) + k.spec(k.c);
            f = k.colfft(axis, k.c + k.s) + 36.0 * k.Vh;
          } else {
            b = 2 * k.spec(k.c);
            f = k.colfft(axis, 2 * k.c) + 100.0 * k.Vh;
          }
        },
        by, fl);
    const int kind = OP == OP_FWD ? KK_COL_FWD : OP == OP_INV ? KK_COL_INV
                   : OP == OP_GRAD ? KK_COL_GRAD : (OP == OP_DIV ? KK_COL_DIV : KK_COL_PREC);
    prof_launch(prec_of<T>(), kind, by, fl, st,
                [&] { k_col256<OP, BXC, B><<<grid, 16 * BXC, sm, st>>>(d, ba, axis); });
  }
}

template <typename T, int OP, int BX, int B>
static void launch_colop_bx(const Launch<T, B>& L, int axis, cudaStream_t st) {
  const int cls = geo_col(axis, OP);
  const int nb = L.grid(cls);
  const size_t sm = L.smem(cls);
  const BatchArgs<T> ba = L.args(cls);
  const Desc<T>* d = L.P.d;
  const bool d3 = L.P.h.ndim == 3;
  double by, fl;
  L.cost(
      [&](const Plan<T>& Q, double& b, double& f) {
        const Cost<T> k(Q.h);
        if (OP == OP_GRAD) {
          b = k.spec(k.c) + k.spec(k.s);
          f = k.colfft(axis, k.c + k.s) + (d3 ? 42.0 : 20.0) * k.Vh;
        } else if (OP == OP_DIV) {
          b = k.spec(k.s) + k.spec(k.c);
          f = k.colfft(axis, k.c + k.s) + (d3 ? 36.0 : 16.0) * k.Vh;
        } else {
          b = 2 * k.spec(k.c);
          f = k.colfft(axis, 2 * k.c) + (d3 ? 100.0 : 40.0) * k.Vh;
        }
      },
      by, fl);
  const int kind = OP == OP_GRAD ? KK_COL_GRAD : (OP == OP_DIV ? KK_COL_DIV : KK_COL_PREC);
  // slots: c (2 or 3) for the preconditioner, s (3 or 6) for gradient / divergence
  constexpr int kSmall = OP == OP_PREC ? 2 : 3;
  constexpr int kLarge = OP == OP_PREC ? 3 : 6;
  // 3-D single-instance FP32 passes over a pure radix-16 axis: the variant without the
  // other stage kinds
  const AxisPlan& ap = L.P.h.ax[axis];
  const bool only16 = ap.cnt[6] > 0 && !ap.cnt[0] && !ap.cnt[1] && !ap.cnt[2] && !ap.cnt[3] && !ap.cnt[4] &&
                      !ap.cnt[5] && !ap.prime;
  prof_launch(prec_of<T>(), kind, by, fl, st, [&] {
    if (!d3)
      k_colop<T, OP, BX, kSmall, B><<<nb, kColThreadsOp, sm, st>>>(d, ba, axis);
    else if constexpr (B == 0 && sizeof(T) == 4) {
      if (only16)
        k_colop<T, OP, BX, kLarge, B, true><<<nb, kColThreadsOp, sm, st>>>(d, ba, axis);
      else
        k_colop<T, OP, BX, kLarge, B><<<nb, kColThreadsOp, sm, st>>>(d, ba, axis);
    } else {
      k_colop<T, OP, BX, kLarge, B><<<nb, kColThreadsOp, sm, st>>>(d, ba, axis);
    }
  });
}

template <typename T, int OP, int B>
static void launch_colop(const Launch<T, B>& L, int axis, cudaStream_t st) {
  switch (L.bx(axis, OP)) {
    case kColReg | 16: launch_col256<T, OP, 16, B>(L, axis, 1, st); break;
    case kColReg | 8: launch_col256<T, OP, 8, B>(L, axis, 1, st); break;
    case kColReg | 4: launch_col256<T, OP, 4, B>(L, axis, 1, st); break;
    case 4: launch_colop_bx<T, OP, 4, B>(L, axis, st); break;
    case 2: launch_colop_bx<T, OP, 2, B>(L, axis, st); break;
    default: launch_colop_bx<T, OP, 1, B>(L, axis, st); break;
  }
}

template <typename T, int B>
static void launch_col_one(const Launch<T, B>& L, int op, int axis, int ncomp, cudaStream_t st);

// A grouped column pass runs one launch per column-tile width among its instances.
template <typename T, int B>
static void launch_col(const Launch<T, B>& L, int op, int axis, int ncomp, cudaStream_t st) {
  if (B == 0 || !L.bl) {
    launch_col_one<T, B>(L, op, axis, ncomp, st);
    return;
  }
  const int cls = geo_col(axis, op);
  for (const ColGroup<T>& g : L.bl->cols[cls - GEO_COL0]) {
    if (g.total == 0) continue;
    BatchLaunch<T> v = *L.bl;
    v.start[cls] = g.start;
    v.total[cls] = g.total;
    v.sm[cls] = g.sm;
    v.bx[axis][op] = g.bx;
    v.plans = g.plans;
    const Launch<T, B> Lg{L.P, &v};
    launch_col_one<T, B>(Lg, op, axis, ncomp, st);
  }
}

template <typename T, int B>
static void launch_col_one(const Launch<T, B>& L, int op, int axis, int ncomp, cudaStream_t st) {
  if (op == OP_FWD || op == OP_INV) {
    switch (L.bx(axis, op)) {
      case kColReg | 16:
        if (op == OP_FWD) launch_col256<T, OP_FWD, 16, B>(L, axis, ncomp, st);
        else launch_col256<T, OP_INV, 16, B>(L, axis, ncomp, st);
        break;
      case kColReg | 8:
        if (op == OP_FWD) launch_col256<T, OP_FWD, 8, B>(L, axis, ncomp, st);
        else launch_col256<T, OP_INV, 8, B>(L, axis, ncomp, st);
        break;
      case kColReg | 4:
        if (op == OP_FWD) launch_col256<T, OP_FWD, 4, B>(L, axis, ncomp, st);
        else launch_col256<T, OP_INV, 4, B>(L, axis, ncomp, st);
        break;
      case 16:
        if constexpr (sizeof(T) == 4) launch_colplain_bx<T, 16, B>(L, op, axis, ncomp, st);
        break;
      case 8: launch_colplain_bx<T, 8, B>(L, op, axis, ncomp, st); break;
      case 4: launch_colplain_bx<T, 4, B>(L, op, axis, ncomp, st); break;
      case 2: launch_colplain_bx<T, 2, B>(L, op, axis, ncomp, st); break;
      default: launch_colplain_bx<T, 1, B>(L, op, axis, ncomp, st); break;
    }
    return;
  }
  if (op == OP_GRAD) launch_colop<T, OP_GRAD, B>(L, axis, st);
  else if (op == OP_DIV) launch_colop<T, OP_DIV, B>(L, axis, st);
  else launch_colop<T, OP_PREC, B>(L, axis, st);
}

// The FP32 x inverse and middle passes of a single-instance launch stage their
// elementwise inputs in shared memory when N1 % 16 == 0 (16-byte runs of every
// staged array) and the staged slot is 16-byte aligned.
template <typename T, int B>
static bool x_stage_ok(const Launch<T, B>& L) {
  return B == 0 && sizeof(T) == 4 && (L.P.h.n1 % 16) == 0;
}

template <typename T, int B>
static void launch_xinv(const Launch<T, B>& L, int post, int in_slot, int out_slot, int masked, int want_dot,
                        cudaStream_t st) {
  const int pi = prec_of<T>();
  const int nb = L.grid(GEO_X);
  size_t sm = L.smem(GEO_X);
  int stage = 0;
  if (x_stage_ok(L) && post != POST_RESID &&
      (post != POST_APPLY || reinterpret_cast<uintptr_t>(L.P.h.slot[in_slot]) % 16 == 0)) {
    const Desc<T>& D = L.P.h;
    stage = 1;
    sm = stage_round(sm) + xinv_stage_layout(post, D.c, D.lx, D.n1, D.phase != nullptr).total;
  }
  const BatchArgs<T> ba = L.args(GEO_X);
  const Desc<T>* d = L.P.d;
  double by, fl;
  L.cost(
      [&](const Plan<T>& Q, double& b, double& f) {
        const Cost<T> k(Q.h);
        const double in = k.spec(k.c), mat = (Q.h.phase ? 2.0 : 0.0) * k.V + k.V;
        f = k.xfft(k.c);
        if (post == POST_APPLY) {
          b = in + 2 * k.real(k.c) + mat;
          f += 2 * k.c * k.V;
        } else if (post == POST_RESID) {
          b = in + 24 * k.c * k.V + mat;
          f += 3 * k.c * k.V;
        } else if (post == POST_PREC_PUPD) {
          b = 2 * in + 2 * k.real(k.c) + k.V;
          f = 2 * k.xfft(k.c) + 2 * k.c * k.V;
        } else {
          b = in + k.real(k.c) + k.V;
        }
      },
      by, fl);
  if constexpr (B == 0 && sizeof(T) == 4) {
    if (L.P.g.xreg && (post == POST_APPLY || post == POST_PREC_PUPD)) {
      const Desc<T>& D = L.P.h;
      const int lx = D.lx;
      size_t smr = xreg_smem(3 * lx / 2);
      if (post == POST_APPLY)
        prof_launch(pi, KK_XINV_APPLY, by, fl, st, [&] {
          k_xinv256<POST_APPLY, B><<<nb, 24 * lx, smr + (stage ? xinv_stage_layout(POST_APPLY, 3, lx, 256,
                                                                                         D.phase != nullptr).total : 0),
                                     st>>>(d, ba, in_slot, out_slot, masked, want_dot, stage);
        });
      else
        prof_launch(pi, KK_XINV_PUPD, by, fl, st, [&] {
          k_xinv256<POST_PREC_PUPD, B><<<nb, 24 * lx, smr, st>>>(d, ba, in_slot, out_slot, masked, 0, 0);
        });
      return;
    }
  }
  switch (post) {
    case POST_APPLY:
      prof_launch(pi, KK_XINV_APPLY, by, fl, st, [&] {
        k_xinv<T, POST_APPLY, B><<<nb, 256, sm, st>>>(d, ba, in_slot, out_slot, masked, want_dot, stage);
      });
      break;
    case POST_RESID:
      prof_launch(pi, KK_XINV_RESID, by, fl, st, [&] {
        k_xinv<T, POST_RESID, B><<<nb, 256, sm, st>>>(d, ba, in_slot, out_slot, masked, want_dot, 0);
      });
      break;
    case POST_PREC_PUPD:
      if constexpr (B == 0)
        prof_launch(pi, KK_XINV_PUPD, by, fl, st, [&] {
          k_xinv<T, POST_PREC_PUPD, B><<<nb, 256, sm, st>>>(d, ba, in_slot, out_slot, masked, 0, stage);
        });
      break;
    default:
      prof_launch(pi, KK_XINV_PREC, by, fl, st,
                  [&] { k_xinv<T, POST_PREC, B><<<nb, 256, sm, st>>>(d, ba, in_slot, out_slot, masked, 0, stage); });
      break;
  }
}

template <typename T, int B>
static void launch_xmid(const Launch<T, B>& L, cudaStream_t st) {
  const int nb = L.grid(GEO_XM);
  size_t sm = L.smem(GEO_XM);
  int stage = 0;
  if (x_stage_ok(L) && L.P.h.phase) {
    stage = 1;
    sm = stage_round(sm) + stage_round((size_t)L.P.h.lxm * L.P.h.n1 * 2);
  }
  const BatchArgs<T> ba = L.args(GEO_XM);
  const Desc<T>* d = L.P.d;
  double by, fl;
  L.cost(
      [&](const Plan<T>& Q, double& b, double& f) {
        const Cost<T> k(Q.h);
        b = 2 * k.spec(k.s) + (Q.h.phase ? 2.0 : 0.0) * k.V;
        f = 2 * k.xfft(k.s) + (Q.h.ndim == 3 ? 66.0 : 15.0) * k.V;
      },
      by, fl);
  if constexpr (B == 0 && sizeof(T) == 4) {
    if (L.P.g.xreg) {
      const int lxm = L.P.h.lxm;
      prof_launch(prec_of<T>(), KK_XMID, by, fl, st,
                  [&] { k_xmid256<B><<<nb, 48 * lxm, xreg_smem_mid(lxm), st>>>(d, ba); });
      return;
    }
  }
  prof_launch(prec_of<T>(), KK_XMID, by, fl, st, [&] { k_xmid<T, B><<<nb, 256, sm, st>>>(d, ba, stage); });
}

template <typename T, int B>
void launch_apply_impl(const Plan<T>& P, int pre, int in_slot, int post, int out_slot, int masked, int want_dot,
                       cudaStream_t st, const BatchLaunch<T>* bl) {
  const Desc<T>& D = P.h;
  const Launch<T, B> L{P, bl};
  if (pre != PRE_NONE) launch_xfwd<T, B>(L, pre, in_slot, st);  // PRE_NONE: the spectrum of in_slot is in place
  if (D.midAxis) launch_col<T, B>(L, OP_FWD, D.midAxis, D.c, st);
  launch_col<T, B>(L, OP_GRAD, D.opAxis, D.c, st);
  if (D.midAxis) launch_col<T, B>(L, OP_INV, D.midAxis, D.s, st);
  launch_xmid<T, B>(L, st);
  if (D.midAxis) launch_col<T, B>(L, OP_FWD, D.midAxis, D.s, st);
  launch_col<T, B>(L, OP_DIV, D.opAxis, D.c, st);
  if (D.midAxis) launch_col<T, B>(L, OP_INV, D.midAxis, D.c, st);
  // PRE_PUPD writes p; the epilogue reads the operator's input from in_slot
  launch_xinv<T, B>(L, post, pre == PRE_PUPD ? (int)SL_P : in_slot, out_slot, masked, want_dot, st);
}

template <typename T, int B>
void launch_precond_impl(const Plan<T>& P, int pre, int in_slot, int out_slot, int masked, cudaStream_t st,
                         const BatchLaunch<T>* bl) {
  const Desc<T>& D = P.h;
  const Launch<T, B> L{P, bl};
  launch_xfwd<T, B>(L, pre, in_slot, st);
  if (D.midAxis) launch_col<T, B>(L, OP_FWD, D.midAxis, D.c, st);
  launch_col<T, B>(L, OP_PREC, D.opAxis, D.c, st);
  if (D.midAxis) launch_col<T, B>(L, OP_INV, D.midAxis, D.c, st);
  launch_xinv<T, B>(L, POST_PREC, in_slot, out_slot, masked, 0, st);
}

template <typename T>
void launch_precond_part_impl(const Plan<T>& P, int part, int pre, int in_slot, int masked, cudaStream_t st) {
  const Desc<T>& D = P.h;
  const Launch<T, 0> L{P, nullptr};
  if (part == 0) {
    launch_xfwd<T, 0>(L, pre, in_slot, st);
    if (D.midAxis) launch_col<T, 0>(L, OP_FWD, D.midAxis, D.c, st);
    launch_col<T, 0>(L, OP_PREC, D.opAxis, D.c, st);
  } else {
    if (D.midAxis) launch_col<T, 0>(L, OP_INV, D.midAxis, D.c, st);
    launch_xinv<T, 0>(L, POST_PREC_PUPD, SL_P, SL_P, masked, 0, st);
  }
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
      packed<T>(buf, row_stride(N), q, x) = line < nsp ? f[(long long)k * D.V + line * N + x] : (T)0;
    }
    __syncthreads();
    fft_lines<T, 1>(buf, D.ax[0], LX * nc / 2, row_stride(N), tw, -1);
    store_unpacked<T>(D, buf, row_stride(N), LX * nc, l0, nc, nsp);
  } else {
    load_packed<T>(D, buf, row_stride(N), LX * nc, l0, nc, nsp);
    __syncthreads();
    fft_lines<T, 1>(buf, D.ax[0], LX * nc / 2, row_stride(N), tw, +1);
    for (int e = threadIdx.x; e < LX * nc * N; e += blockDim.x) {
      const int x = e % N, q = e / N, k = q % nc, l = q / nc;
      const long long line = l0 + l;
      if (line < nsp) f[(long long)k * D.V + line * N + x] = packed<T>(buf, row_stride(N), q, x);
    }
  }
}

// x lines per block of the standalone transform of ncomp components, and whether its
// tile fits (ncomp = 5 in 3-D takes five line pairs per tile on long x axes).
template <typename T>
int rfft3_lines(const Plan<T>& P, int ncomp) {
  const Desc<T>& D = P.h;
  const int ex = std::min(2048, max_tile_elems<T>(D.ax[0], P.g.thr));
  return x_tile_lines(D.n1, (long long)D.n2 * D.n3, ex, ncomp);
}
template <typename T>
bool rfft3_fits(const Plan<T>& P, int ncomp) {
  return x_tile_fits(P.h, P.g.thr, rfft3_lines(P, ncomp), ncomp);
}
template <typename T>
int axis_tile_capacity(const AxisPlan& pl) {
  return max_tile_elems<T>(pl, 256);
}

template <typename T>
void launch_rfft3(const Plan<T>& P, int dir, int ncomp, int real_slot, cudaStream_t st) {
  const Desc<T>& D = P.h;
  const PassGeo& g = P.g;
  const long long nsp = (long long)D.n2 * D.n3;
  const int lx = rfft3_lines(P, ncomp);
  const int nb = (int)((nsp + lx - 1) / lx);
  const size_t sm = (size_t)(D.n1 + (lx * ncomp / 2) * row_stride(D.n1)) * sizeof(cplx<T>);
  const int axes[2] = {1, 2};
  const Launch<T, 0> L{P, nullptr};
  if (dir < 0) {
    prof_launch(prec_of<T>(), KK_XFWD_PLAIN, Cost<T>(D).real(ncomp) + Cost<T>(D).spec(ncomp),
                Cost<T>(D).xfft(ncomp), st, [&] { k_xplain<T><<<nb, g.thr, sm, st>>>(P.d, lx, ncomp, -1, real_slot); });
    for (int a : axes)
      if ((a == 1 ? D.n2 : D.n3) > 1) launch_col<T, 0>(L, OP_FWD, a, ncomp, st);
  } else {
    for (int a : {2, 1})
      if ((a == 1 ? D.n2 : D.n3) > 1) launch_col<T, 0>(L, OP_INV, a, ncomp, st);
    prof_launch(prec_of<T>(), KK_XINV_PREC, Cost<T>(D).real(ncomp) + Cost<T>(D).spec(ncomp),
                Cost<T>(D).xfft(ncomp), st, [&] { k_xplain<T><<<nb, g.thr, sm, st>>>(P.d, lx, ncomp, +1, real_slot); });
  }
}

template <typename T, int B>
cudaError_t init_kernel_attributes_impl() {
  const int maxsm = 200 * 1024;  // opt-in limit minus the static shared memory of the reductions
  cudaError_t e = cudaSuccess;
#define WFFT_SETATTR(k)                                                                    \
  do {                                                                                     \
    cudaError_t ee = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm); \
    if (ee != cudaSuccess) e = ee;                                                         \
  } while (0)
  WFFT_SETATTR((k_xfwd<T, PRE_PLAIN, B>));
  WFFT_SETATTR((k_xfwd<T, PRE_PUPD, B>));
  WFFT_SETATTR((k_xfwd<T, PRE_RUPD, B>));
  WFFT_SETATTR((k_xfwd<T, PRE_CONV, B>));
  WFFT_SETATTR((k_xfwd<T, PRE_XUPD, B>));
  if constexpr (B == 0 && sizeof(T) == 4) WFFT_SETATTR((k_xfwd<T, PRE_CONVD, B>));
  WFFT_SETATTR((k_xinv<T, POST_APPLY, B>));
  WFFT_SETATTR((k_xinv<T, POST_RESID, B>));
  WFFT_SETATTR((k_xinv<T, POST_PREC, B>));
  if constexpr (B == 0) WFFT_SETATTR((k_xinv<T, POST_PREC_PUPD, B>));
  WFFT_SETATTR((k_xmid<T, B>));
  if constexpr (B == 0 && sizeof(T) == 4) {
    WFFT_SETATTR((k_xmid256<B>));
    WFFT_SETATTR((k_xinv256<POST_APPLY, B>));
    WFFT_SETATTR((k_xinv256<POST_PREC_PUPD, B>));
    WFFT_SETATTR((k_xfwd256_rupd<B>));
  }
  if (!B) WFFT_SETATTR((k_xplain<T>));
#define WFFT_SETATTR_BX(BXV)                  \
  WFFT_SETATTR((k_colop<T, OP_GRAD, BXV, 3, B>));  \
  WFFT_SETATTR((k_colop<T, OP_GRAD, BXV, 6, B>));  \
  WFFT_SETATTR((k_colop<T, OP_DIV, BXV, 3, B>));   \
  WFFT_SETATTR((k_colop<T, OP_DIV, BXV, 6, B>));   \
  WFFT_SETATTR((k_colop<T, OP_PREC, BXV, 2, B>));  \
  WFFT_SETATTR((k_colop<T, OP_PREC, BXV, 3, B>));
  WFFT_SETATTR_BX(1)
  WFFT_SETATTR_BX(2)
  WFFT_SETATTR_BX(4)
  if constexpr (B == 0 && sizeof(T) == 4) {
#define WFFT_SETATTR_R16(BXV)                             \
  WFFT_SETATTR((k_colop<T, OP_GRAD, BXV, 6, B, true>)); \
  WFFT_SETATTR((k_colop<T, OP_DIV, BXV, 6, B, true>));  \
  WFFT_SETATTR((k_colop<T, OP_PREC, BXV, 3, B, true>));
    WFFT_SETATTR_R16(1)
    WFFT_SETATTR_R16(2)
    WFFT_SETATTR_R16(4)
  }
  WFFT_SETATTR((k_colplain<T, OP_FWD, 1, B>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 1, B>));
  WFFT_SETATTR((k_colplain<T, OP_FWD, 2, B>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 2, B>));
  WFFT_SETATTR((k_colplain<T, OP_FWD, 4, B>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 4, B>));
  WFFT_SETATTR((k_colplain<T, OP_FWD, 8, B>));
  WFFT_SETATTR((k_colplain<T, OP_INV, 8, B>));
  if constexpr (sizeof(T) == 4) {
    WFFT_SETATTR((k_colplain<T, OP_FWD, 16, B>));
    WFFT_SETATTR((k_colplain<T, OP_INV, 16, B>));
#define WFFT_SETATTR_REG(BXC)                \
  WFFT_SETATTR((k_col256<OP_FWD, BXC, B>));  \
  WFFT_SETATTR((k_col256<OP_INV, BXC, B>));  \
  WFFT_SETATTR((k_col256<OP_GRAD, BXC, B>)); \
  WFFT_SETATTR((k_col256<OP_DIV, BXC, B>));  \
  WFFT_SETATTR((k_col256<OP_PREC, BXC, B>));
    WFFT_SETATTR_REG(4)
    WFFT_SETATTR_REG(8)
    WFFT_SETATTR_REG(16)
#undef WFFT_SETATTR_REG
  }
#undef WFFT_SETATTR_BX
#undef WFFT_SETATTR
  return e;
}

// Single-instance kernels and the shared host helpers.
#define WFFT_INSTANTIATE(T)                                                                                  \
  template void plan_geometry<T>(Plan<T>&);                                                                  \
  template bool col_bx_feasible<T>(const Plan<T>&, int, int, int);                                          \
  template void set_col_bx<T>(Plan<T>&, int, int, int);                                                     \
  template void launch_apply_impl<T, 0>(const Plan<T>&, int, int, int, int, int, int, cudaStream_t,          \
                                        const BatchLaunch<T>*);                                              \
  template void launch_precond_impl<T, 0>(const Plan<T>&, int, int, int, int, cudaStream_t,                  \
                                          const BatchLaunch<T>*);                                            \
  template void launch_precond_part_impl<T>(const Plan<T>&, int, int, int, int, cudaStream_t);              \
  template int geo_blocks<T>(const Plan<T>&, int, int);                                                     \
  template size_t geo_smem<T>(const Plan<T>&, int, int);                                                    \
  template void launch_rfft3<T>(const Plan<T>&, int, int, int, cudaStream_t);                               \
  template bool rfft3_fits<T>(const Plan<T>&, int);                                                         \
  template int axis_tile_capacity<T>(const AxisPlan&);                                                      \
  template cudaError_t init_kernel_attributes_impl<T, 0>();

// Grouped (batched) kernels.
#define WFFT_INSTANTIATE_BATCH(T)                                                                            \
  template void launch_apply_impl<T, 1>(const Plan<T>&, int, int, int, int, int, int, cudaStream_t,          \
                                        const BatchLaunch<T>*);                                              \
  template void launch_precond_impl<T, 1>(const Plan<T>&, int, int, int, int, cudaStream_t,                  \
                                          const BatchLaunch<T>*);                                            \
  template cudaError_t init_kernel_attributes_impl<T, 1>();

}  // namespace wfft
