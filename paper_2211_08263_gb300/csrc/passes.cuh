// Pass kernels of the spectral operator and preconditioner.
//
// A 3-D real field goes through the half spectrum as
//   x pass (real <-> complex along x_1, two real lines packed per complex line)
//   y pass (complex along x_2), z pass (complex along x_3),
// and the pointwise work of the method is fused into these passes:
//   * operator A of Eq. Fourier_ND_A:
//       xfwd(p) -> y fwd -> z[fwd, eps^ = sym(i xi (x) u^), inv] -> y inv
//       -> x[inv, sigma = C(x) : eps, fwd] -> y fwd -> z[fwd, t^ = i xi . sigma^, inv]
//       -> y inv -> xinv[q = -theta t + rho p, mask]
//   * preconditioner of Eq. precond / Eq. acous:
//       xfwd(r) -> y fwd -> z[fwd, z^ = (theta K(xi) + rho_bar I)^-1 r^, inv] -> y inv -> xinv[mask]
//   * Krylov vector updates (x += alpha p, r -= alpha q, p = z + beta p), the
//     Fourier-space (r, z) by Parseval and (p, q), ||r||^2 as FP64 block partial sums.
// In 2-D (N3 = 1) the y pass hosts the spectral multiply and there is no
// middle pass.  Strains are engineering (gamma_ij = 2 eps_ij, Voigt order
// 11,22,33,23,13,12; 2-D: 11,22,12) so sigma = Cv e with the Voigt matrix Cv.
// The DFT is unnormalised; 1/V is folded into the spectral multiplies.
#pragma once
#include "common.cuh"
#include "fft_core.cuh"

namespace wfft {

enum { PRE_PLAIN = 0, PRE_PUPD = 1, PRE_RUPD = 2, PRE_CONV = 3, PRE_XUPD = 4, PRE_CONVD = 5, PRE_NONE = 6 };
enum { POST_APPLY = 0, POST_RESID = 1, POST_PREC = 2, POST_PREC_PUPD = 3 };
enum { OP_FWD = 0, OP_INV = 1, OP_GRAD = 2, OP_DIV = 3, OP_PREC = 4 };

template <typename T>
__device__ __forceinline__ T rho_at(const Desc<T>& D, long long vox) {
  return D.rhotab[D.phase ? (long long)D.phase[vox] : vox];
}

// Element x of real line q (pair q/2, part q&1) of a packed buffer.
template <typename T>
__device__ __forceinline__ T& packed(cplx<T>* buf, int lstr, int q, int x) {
  return reinterpret_cast<T*>(buf + (size_t)(q >> 1) * lstr + rowpad(x))[q & 1];
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
__device__ __forceinline__ int num_warps() { return blockDim.x >> 5; }

// Split the complex FFT of two packed real lines into their half spectra and
// store them: A = (Z_k + conj Z_{N-k})/2, B = (Z_k - conj Z_{N-k})/(2i).
// One warp per pair of lines, lanes along kx (no integer division per element).
template <typename T>
__device__ __forceinline__ void store_unpacked(const Desc<T>& D, const cplx<T>* buf, int lstr, int nlines_real,
                                               long long l0, int nc, long long nsp) {
  const int N = D.n1, nh = D.nh;
  const int npairs = nlines_real >> 1;
  for (int p = warp_id(); p < npairs; p += num_warps()) {
    const int qa = 2 * p, qb = 2 * p + 1;
    const long long la = l0 + qa / nc, lb = l0 + qb / nc;
    cplx<T>* da = D.spec + (long long)(qa % nc) * D.Vh + la * D.pitch;
    cplx<T>* db = D.spec + (long long)(qb % nc) * D.Vh + lb * D.pitch;
    const cplx<T>* row = buf + (size_t)p * lstr;
    for (int kx = lane_id(); kx < nh; kx += 32) {
      const cplx<T> Z = row[rowpad(kx)];
      const cplx<T> W = row[rowpad(kx == 0 ? 0 : N - kx)];
      const T h = (T)0.5;
      if (la < nsp) da[kx] = cmake<T>((Z.x + W.x) * h, (Z.y - W.y) * h);
      if (lb < nsp) db[kx] = cmake<T>((Z.y + W.y) * h, (W.x - Z.x) * h);
    }
  }
}

// Load the half spectra of two real lines per complex line as Z = A + i B
// over the full length (Hermitian extension); DC and Nyquist take real parts.
// Load the half spectra of two real lines per complex line as Z = A + i B
// over the full length (Hermitian extension); DC and Nyquist take real parts.
// One warp per pair of lines; each lane keeps 4 kx loads of both lines in flight.
template <typename T>
__device__ __forceinline__ void load_packed(const Desc<T>& D, cplx<T>* buf, int lstr, int nlines_real, long long l0,
                                            int nc, long long nsp) {
  constexpr int U = 4;
  const int N = D.n1, nh = D.nh;
  const int npairs = nlines_real >> 1;
  for (int p = warp_id(); p < npairs; p += num_warps()) {
    const int qa = 2 * p, qb = 2 * p + 1;
    const long long la = l0 + qa / nc, lb = l0 + qb / nc;
    const cplx<T>* sa = D.spec + (long long)(qa % nc) * D.Vh + la * D.pitch;
    const cplx<T>* sb = D.spec + (long long)(qb % nc) * D.Vh + lb * D.pitch;
    cplx<T>* row = buf + (size_t)p * lstr;
    // the Nyquist column of an even N is taken by lane 0 next to kx = 0, so that
    // the main loop covers exactly N/2 columns (one pass of 32 U for N = 256)
    const int nk = (N & 1) ? nh : nh - 1;
    const bool ny = !(N & 1) && lane_id() == 0;
    cplx<T> An = cmake<T>(0, 0), Bn = cmake<T>(0, 0);
    if (ny) {
      if (la < nsp) An = sa[N / 2];
      if (lb < nsp) Bn = sb[N / 2];
    }
    for (int k0 = lane_id(); k0 < nk; k0 += 32 * U) {
      cplx<T> A[U], B[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kx = k0 + 32 * u;
        A[u] = (kx < nk && la < nsp) ? sa[kx] : cmake<T>(0, 0);
        B[u] = (kx < nk && lb < nsp) ? sb[kx] : cmake<T>(0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int kx = k0 + 32 * u;
        if (kx >= nk) continue;
        if (kx == 0) {
          row[rowpad(0)] = cmake<T>(A[u].x, B[u].x);
        } else {
          row[rowpad(kx)] = cmake<T>(A[u].x - B[u].y, A[u].y + B[u].x);
          row[rowpad(N - kx)] = cmake<T>(A[u].x + B[u].y, B[u].x - A[u].y);
        }
      }
    }
    if (ny) row[rowpad(N / 2)] = cmake<T>(An.x, Bn.x);
  }
}

// ---------------------------------------------------------------------------
// Staging of the elementwise inputs of the FP32 x passes: the rows a block's epilogue
// (or Hooke phase) reads are copied global -> shared with cp.async at the start of the
// block, so they arrive while the spectrum is loaded and transformed, with every byte
// of the block in flight at once.  A block's LX lines of one component are one
// contiguous run of LX N elements, so each staged array is one run per component.
// Staging needs N % 16 == 0 (16-byte runs for 1-byte masks); the host decides and
// sizes the shared memory (stage != 0).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ size_t stage_round(size_t b) { return (b + 15) & ~(size_t)15; }

// Byte layout of the staging area of an x inverse pass: p (POST_APPLY: the operator's
// input; POST_PREC_PUPD: the previous search direction; nc x LX x N floats), rho source
// (POST_APPLY: LX x N uint16 phase ids, or floats of per-voxel rho), mask (LX x N bytes).
struct XStage {
  size_t p, rho, mask, total;
};
__host__ __device__ __forceinline__ XStage xinv_stage_layout(int post, int nc, int LX, int N, bool phase) {
  XStage L;
  const size_t e = (size_t)LX * N;
  const bool wp = post == POST_APPLY || post == POST_PREC_PUPD, wr = post == POST_APPLY;
  L.p = 0;
  L.rho = stage_round(wp ? (size_t)nc * e * 4 : 0);
  L.mask = L.rho + stage_round(wr ? e * (phase ? 2 : 4) : 0);
  L.total = L.mask + stage_round(e);
  return L;
}

// Issue 16-byte cp.async copies of `bytes` (a multiple of 16, both ends 16-byte aligned).
__device__ __forceinline__ void stage_copy(void* sdst, const void* gsrc, size_t bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const char* g = reinterpret_cast<const char*>(gsrc);
  for (size_t o = (size_t)threadIdx.x * 16; o < bytes; o += (size_t)blockDim.x * 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s + (unsigned)o), "l"(g + o) : "memory");
}
__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Waits for this thread's own copies only (they complete unconditionally); a barrier
// after it makes every thread's copies visible to the block.
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ void load_twiddles(cplx<T>* tw, const cplx<T>* src, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = src[i];
}

// ---------------------------------------------------------------------------
// x forward pass: real c-component field -> half spectrum, with fused updates
//   PRE_PLAIN  input slot in_slot
//   PRE_PUPD   p = z + beta p (p = z on the first iteration)
//   PRE_RUPD   r -= alpha q, ||r||^2, and the solution update: x += alpha p (FP64
//              solve) or d += alpha p (FP32 correction of a mixed inner solve)
//   PRE_CONV   r = scale * r64 in T, d = 0 (start of a mixed inner solve)
//   PRE_CONVD  r = scale * (r64 - q), d = scale * d (start of a mixed inner solve
//              from the initial guess d with q = P A d already formed)
//   PRE_XUPD   x += xcoef * d (FP64 descriptor of a mixed solve: folds the
//              finished inner correction into the FP64 solution) and transform x
// ---------------------------------------------------------------------------
template <typename T, int PRE, int BATCH>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 4) k_xfwd(const Desc<T>* __restrict__ dd, BatchArgs<T> ba, int in_slot) {
  int blk;
  const Desc<T>* __restrict__ Dp = pick_ptr<T, BATCH>(dd, ba, blk);
  const Desc<T>& D = *Dp;
  const int LX = D.lx;
  Scalars* sc = D.sc;
  if (sc->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = D.n1, nc = D.c;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* buf = tw + N;
  const int lstr = row_stride(N);
  const long long nsp = (long long)D.n2 * D.n3;
  const long long l0 = (long long)blk * LX;
  const long long V = D.V;
  load_twiddles<T>(tw, D.tw[0], N);
  bool first = false;
  T beta = 0, alpha = 0;
  double scale = 1.0, xc = 0.0;
  if (PRE == PRE_PUPD) {
    first = sc->first != 0;
    beta = (T)sc->beta;
  }
  if (PRE == PRE_RUPD) alpha = (T)sc->alpha;
  if (PRE == PRE_CONV || PRE == PRE_CONVD) scale = sc->scale;
  if (PRE == PRE_XUPD) xc = D.sc_inner->xcoef;
  DotAcc<T> acc;
  constexpr int U = 4;  // elements per lane kept in flight
  const int nq = LX * nc;
  // work items (line, chunk of 32 U elements) spread evenly over the warps
  const int nch = (N + 32 * U - 1) / (32 * U);
  for (int it = warp_id(); it < nq * nch; it += num_warps()) {
    const int q = it / nch;
    const int k = q % nc, l = q / nc;
    const long long line = l0 + l;
    const bool valid = line < nsp;
    const long long g0 = (long long)k * V + line * N;
    {
      const int x0 = (it - q * nch) * 32 * U + lane_id();
      T a[U], b[U], c[U], e[U];
      double w[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int x = x0 + 32 * u;
        const bool ok = valid && x < N;
        const long long gi = g0 + x;
        a[u] = b[u] = c[u] = e[u] = 0;
        w[u] = 0.0;
        if (ok) {
          if (PRE == PRE_PLAIN) {
            a[u] = reinterpret_cast<const T*>(D.slot[in_slot])[gi];
          } else if (PRE == PRE_PUPD) {
            a[u] = reinterpret_cast<const T*>(D.slot[SL_Z])[gi];
            if (!first) b[u] = reinterpret_cast<const T*>(D.slot[SL_P])[gi];
          } else if (PRE == PRE_RUPD) {
            a[u] = reinterpret_cast<const T*>(D.slot[SL_P])[gi];
            b[u] = reinterpret_cast<const T*>(D.slot[SL_Q])[gi];
            c[u] = reinterpret_cast<const T*>(D.slot[SL_R])[gi];
            e[u] = sizeof(T) == 8 ? reinterpret_cast<const T*>(D.slot[SL_X])[gi]
                                  : reinterpret_cast<const T*>(D.slot[SL_D])[gi];
          } else if (PRE == PRE_CONV) {
            w[u] = reinterpret_cast<const double*>(D.slot[SL_R64])[gi];
          } else if (PRE == PRE_CONVD) {
            w[u] = reinterpret_cast<const double*>(D.slot[SL_R64])[gi];
            b[u] = reinterpret_cast<const T*>(D.slot[SL_Q])[gi];
            e[u] = reinterpret_cast<const T*>(D.slot[SL_D])[gi];
          } else {  // PRE_XUPD (T = double)
            a[u] = reinterpret_cast<const T*>(D.slot[SL_X])[gi];
            e[u] = (T)reinterpret_cast<const float*>(D.slot[SL_D])[gi];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int x = x0 + 32 * u;
        if (x >= N) continue;
        const bool ok = valid;
        const long long gi = g0 + x;
        T val = 0;
        if (ok) {
          if (PRE == PRE_PLAIN) {
            val = a[u];
          } else if (PRE == PRE_PUPD) {
            val = first ? a[u] : a[u] + beta * b[u];
            reinterpret_cast<T*>(D.slot[SL_P])[gi] = val;
          } else if (PRE == PRE_RUPD) {
            const T sol = e[u] + alpha * a[u];
            if (sizeof(T) == 8)
              reinterpret_cast<T*>(D.slot[SL_X])[gi] = sol;
            else
              reinterpret_cast<T*>(D.slot[SL_D])[gi] = sol;
            val = c[u] - alpha * b[u];
            reinterpret_cast<T*>(D.slot[SL_R])[gi] = val;
            acc.add_prod(val, val);
          } else if (PRE == PRE_CONV) {
            val = (T)(w[u] * scale);
            reinterpret_cast<T*>(D.slot[SL_R])[gi] = val;
            reinterpret_cast<T*>(D.slot[SL_D])[gi] = (T)0;
          } else if (PRE == PRE_CONVD) {
            val = (T)((w[u] - (double)b[u]) * scale);
            reinterpret_cast<T*>(D.slot[SL_R])[gi] = val;
            reinterpret_cast<T*>(D.slot[SL_D])[gi] = (T)((double)e[u] * scale);
          } else {  // PRE_XUPD
            val = a[u] + (T)(xc * (double)e[u]);
            reinterpret_cast<T*>(D.slot[SL_X])[gi] = val;
          }
        }
        packed<T>(buf, lstr, q, x) = val;
      }
    }
  }
  if (PRE == PRE_RUPD) {
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) D.part[PT_A][blk] = s;
  }
  __syncthreads();
  fft_lines<T, 1>(buf, D.ax[0], LX * nc / 2, lstr, tw, -1);
  store_unpacked<T>(D, buf, lstr, LX * nc, l0, nc, nsp);
}

// ---------------------------------------------------------------------------
// x inverse pass: half spectrum -> real field with fused epilogue
//   POST_APPLY  q = t + rho p (t = -theta div sigma), mask, (p, q)
//   POST_RESID  A x = t + rho x (kept when the slot exists), r = P(b - A x), ||r||^2
//   POST_PREC   z = P(t)
//   POST_PREC_PUPD  z = P(t), p = z + beta p (p = z on a solve's first iteration), then
//               the forward x transform of p back into the half spectrum: the next
//               operator application starts at its first column pass (PRE_NONE), and z
//               never goes to memory
// ---------------------------------------------------------------------------
template <typename T, int POST, int BATCH>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 4) k_xinv(const Desc<T>* __restrict__ dd, BatchArgs<T> ba, int in_slot,
                                              int out_slot, int masked, int want_dot, int stage_arg) {
  const int stage = sizeof(T) == 4 ? stage_arg : 0;  // FP32 passes only
  int blk;
  const Desc<T>* __restrict__ Dp = pick_ptr<T, BATCH>(dd, ba, blk);
  const Desc<T>& D = *Dp;
  const int LX = D.lx;
  Scalars* sc = D.sc;
  if (sc->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = D.n1, nc = D.c;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* buf = tw + N;
  const int lstr = row_stride(N);
  const long long nsp = (long long)D.n2 * D.n3;
  const long long l0 = (long long)blk * LX;
  const long long V = D.V;
  // staged epilogue inputs (FP32 passes): issued first, consumed after the FFT
  unsigned char* stg = smraw + stage_round((size_t)(N + (LX * nc / 2) * lstr) * sizeof(cplx<T>));
  const XStage SL = xinv_stage_layout(POST, nc, LX, N, D.phase != nullptr);
  // POST_PREC_PUPD: p = z + beta p needs the old p unless this is the first iteration
  const bool pfirst = POST == POST_PREC_PUPD && sc->first != 0;
  const T pbeta = POST == POST_PREC_PUPD ? (T)sc->beta : (T)0;
  const int pin = POST == POST_PREC_PUPD ? (int)SL_P : in_slot;
  if (stage) {
    const long long nv = nsp - l0 < LX ? nsp - l0 : LX;  // valid lines of this block
    const size_t e = (size_t)nv * N;
    if (POST == POST_APPLY || (POST == POST_PREC_PUPD && !pfirst))
      for (int k = 0; k < nc; ++k)
        stage_copy(stg + SL.p + (size_t)k * LX * N * 4,
                   reinterpret_cast<const float*>(D.slot[pin]) + (long long)k * V + l0 * N, e * 4);
    if (POST == POST_APPLY) {
      if (D.phase)
        stage_copy(stg + SL.rho, D.phase + l0 * N, e * 2);
      else
        stage_copy(stg + SL.rho, D.rhotab + l0 * N, e * 4);
    }
    if (masked) stage_copy(stg + SL.mask, D.mask + l0 * N, e);
    stage_commit();
  }
  load_twiddles<T>(tw, D.tw[0], N);
  load_packed<T>(D, buf, lstr, LX * nc, l0, nc, nsp);
  __syncthreads();
  fft_lines<T, 1>(buf, D.ax[0], LX * nc / 2, lstr, tw, +1);
  if (stage) {
    stage_wait();
    __syncthreads();
  }
  DotAcc<T> acc;
  constexpr int U = 4;  // elements per lane kept in flight
  const int nq = LX * nc;
  // work items (line, chunk of 32 U elements) spread evenly over the warps
  const int nch = (N + 32 * U - 1) / (32 * U);
  for (int it = warp_id(); it < nq * nch; it += num_warps()) {
    const int q = it / nch;
    const int k = q % nc, l = q / nc;
    const long long line = l0 + l;
    if (line >= nsp) continue;
    {
      const int x0 = (it - q * nch) * 32 * U + lane_id();
      T a[U], b[U], rho[U];
      uint8_t m[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int x = x0 + 32 * u;
        a[u] = b[u] = rho[u] = 0;
        m[u] = 0;
        if (x < N && stage) {
          const int ex = l * N + x;  // element of the staged runs
          if (masked) m[u] = stg[SL.mask + ex];
          if (POST == POST_APPLY) {
            a[u] = reinterpret_cast<const T*>(stg + SL.p)[(size_t)k * LX * N + ex];
            rho[u] = D.phase ? D.rhotab[reinterpret_cast<const uint16_t*>(stg + SL.rho)[ex]]
                             : reinterpret_cast<const T*>(stg + SL.rho)[ex];
          } else if (POST == POST_PREC_PUPD && !pfirst) {
            a[u] = reinterpret_cast<const T*>(stg + SL.p)[(size_t)k * LX * N + ex];
          }
        } else if (x < N) {
          const long long vox = line * N + x;
          const long long gi = (long long)k * V + vox;
          if (masked) m[u] = D.mask[vox];
          if (POST == POST_APPLY) {
            a[u] = reinterpret_cast<const T*>(D.slot[in_slot])[gi];
            rho[u] = rho_at<T>(D, vox);
          } else if (POST == POST_PREC_PUPD && !pfirst) {
            a[u] = reinterpret_cast<const T*>(D.slot[SL_P])[gi];
          } else if (POST == POST_RESID) {
            a[u] = reinterpret_cast<const T*>(D.slot[SL_X])[gi];
            b[u] = reinterpret_cast<const T*>(D.slot[SL_B])[gi];
            rho[u] = rho_at<T>(D, vox);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int x = x0 + 32 * u;
        if (x >= N) continue;
        const long long vox = line * N + x;
        const long long gi = (long long)k * V + vox;
        const T t = packed<T>(buf, lstr, q, x);
        const bool isg = (m[u] >> k) & 1;
        if (POST == POST_APPLY) {
          T qv = t + rho[u] * a[u];
          if (isg) qv = 0;
          reinterpret_cast<T*>(D.slot[out_slot])[gi] = qv;
          acc.add_prod(a[u], qv);
        } else if (POST == POST_RESID) {
          const T ax = t + rho[u] * a[u];
          if (D.slot[SL_AU]) reinterpret_cast<T*>(D.slot[SL_AU])[gi] = ax;
          T rv = b[u] - ax;
          if (isg) rv = 0;
          reinterpret_cast<T*>(D.slot[SL_R64])[gi] = rv;
          acc.add_prod(rv, rv);
        } else if (POST == POST_PREC_PUPD) {
          const T z = isg ? (T)0 : t;
          const T pv = pfirst ? z : z + pbeta * a[u];
          reinterpret_cast<T*>(D.slot[SL_P])[gi] = pv;
          packed<T>(buf, lstr, q, x) = pv;
        } else {  // POST_PREC
          reinterpret_cast<T*>(D.slot[out_slot])[gi] = isg ? (T)0 : t;
        }
      }
    }
  }
  if ((POST == POST_APPLY || POST == POST_RESID) && want_dot) {
    const double s = block_sum(acc.value());
    if (threadIdx.x == 0) D.part[PT_A][blk] = s;
  }
  if (POST == POST_PREC_PUPD) {
    __syncthreads();
    fft_lines<T, 1>(buf, D.ax[0], LX * nc / 2, lstr, tw, -1);
    store_unpacked<T>(D, buf, lstr, LX * nc, l0, nc, nsp);
  }
}

// ---------------------------------------------------------------------------
// x middle pass: strain half spectra -> real strains -> sigma = C(x):e -> stress half spectra
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void hooke3(const T* __restrict__ C, T* e) {
  const T e0 = e[0], e1 = e[1], e2 = e[2], e3 = e[3], e4 = e[4], e5 = e[5];
  e[0] = C[0] * e0 + C[1] * e1 + C[2] * e2 + C[3] * e3 + C[4] * e4 + C[5] * e5;
  e[1] = C[1] * e0 + C[6] * e1 + C[7] * e2 + C[8] * e3 + C[9] * e4 + C[10] * e5;
  e[2] = C[2] * e0 + C[7] * e1 + C[11] * e2 + C[12] * e3 + C[13] * e4 + C[14] * e5;
  e[3] = C[3] * e0 + C[8] * e1 + C[12] * e2 + C[15] * e3 + C[16] * e4 + C[17] * e5;
  e[4] = C[4] * e0 + C[9] * e1 + C[13] * e2 + C[16] * e3 + C[18] * e4 + C[19] * e5;
  e[5] = C[5] * e0 + C[10] * e1 + C[14] * e2 + C[17] * e3 + C[19] * e4 + C[20] * e5;
}
template <typename T>
__device__ __forceinline__ void hooke2(const T* __restrict__ C, T* e) {
  const T e0 = e[0], e1 = e[1], e2 = e[2];
  e[0] = C[0] * e0 + C[1] * e1 + C[2] * e2;
  e[1] = C[1] * e0 + C[3] * e1 + C[4] * e2;
  e[2] = C[2] * e0 + C[4] * e1 + C[5] * e2;
}

// One padded stiffness row (24 or 8 values, 16-byte aligned) with vector loads.
template <typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ src, T* dst, int n) {
  if (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (4 * i < n) d4[i] = __ldg(s4 + i);
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int i = 0; i < 12; ++i)
      if (2 * i < n) d2[i] = __ldg(s2 + i);
  }
}

template <typename T, int BATCH>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 4) k_xmid(const Desc<T>* __restrict__ dd, BatchArgs<T> ba,
                                                                        int stage_arg) {
  const int stage = sizeof(T) == 4 ? stage_arg : 0;  // FP32 passes only
  int blk;
  const Desc<T>* __restrict__ Dp = pick_ptr<T, BATCH>(dd, ba, blk);
  const Desc<T>& D = *Dp;
  const int LX = D.lxm;
  if (D.sc->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = D.n1, ns = D.s;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* buf = tw + N;
  const int lstr = row_stride(N);
  const long long nsp = (long long)D.n2 * D.n3;
  const long long l0 = (long long)blk * LX;
  // staged phase ids of the block's voxels (phase tables, FP32 passes)
  const uint16_t* sph =
      reinterpret_cast<const uint16_t*>(smraw + stage_round((size_t)(N + (LX * ns / 2) * lstr) * sizeof(cplx<T>)));
  if (stage) {
    const long long nv = nsp - l0 < LX ? nsp - l0 : LX;
    stage_copy(const_cast<uint16_t*>(sph), D.phase + l0 * N, (size_t)nv * N * 2);
    stage_commit();
  }
  load_twiddles<T>(tw, D.tw[0], N);
  load_packed<T>(D, buf, lstr, LX * ns, l0, ns, nsp);
  __syncthreads();
  fft_lines<T, 1>(buf, D.ax[0], LX * ns / 2, lstr, tw, +1);
  if (stage) {
    stage_wait();
    __syncthreads();
  }
  const int cstride = (ns == 6) ? kCtabStride3 : kCtabStride2;
  // every thread of the block takes voxels (consecutive x across a warp)
  const int lgN = log2_if_pow2(N);
  for (int e = threadIdx.x; e < LX * N; e += blockDim.x) {
    const int l = lgN >= 0 ? e >> lgN : e / N;
    const int x = e - l * N;
    const long long line = l0 + l;
    if (line >= nsp) continue;
    const long long vox = line * N + x;
    const long long row = stage ? (long long)sph[e] : (D.phase ? (long long)D.phase[vox] : vox);
    T C[24];
    load_row<T>(D.ctab + row * cstride, C, ns == 6 ? 24 : 8);
    T ev[6];
    if (ns == 6) {
#pragma unroll
      for (int k = 0; k < 6; ++k) ev[k] = packed<T>(buf, lstr, l * 6 + k, x);
      hooke3<T>(C, ev);
#pragma unroll
      for (int k = 0; k < 6; ++k) packed<T>(buf, lstr, l * 6 + k, x) = ev[k];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) ev[k] = packed<T>(buf, lstr, l * 3 + k, x);
      hooke2<T>(C, ev);
#pragma unroll
      for (int k = 0; k < 3; ++k) packed<T>(buf, lstr, l * 3 + k, x) = ev[k];
    }
  }
  __syncthreads();
  fft_lines<T, 1>(buf, D.ax[0], LX * ns / 2, lstr, tw, -1);
  store_unpacked<T>(D, buf, lstr, LX * ns, l0, ns, nsp);
}

// ---------------------------------------------------------------------------
// column passes (y or z): tiles of BX consecutive kx columns x the full axis.
// The tiles of all components a pass needs sit interleaved in shared memory,
// element (slot t, axis index y, column b) at  y * NS * BX + t * BX + b,  so that
// each kernel runs exactly one forward and one inverse batched FFT over all of
// its lines (line stride 1, element stride NS * BX).
// ---------------------------------------------------------------------------
constexpr int kColThreadsPlain = 256;  // plain transforms (one component per block)
constexpr int kColThreadsOp = 256;     // fused gradient / divergence / preconditioner

// Element stride of a column tile of ns slots x bx columns: ns bx plus a pad for the
// six-slot (3-D gradient / divergence) tiles, chosen so that the FFT stages' reads and
// writes of 3 bx interleaved lines spread over the shared-memory banks (e.g. 24 -> 28
// for bx = 4 in FP32: three wavefronts per warp access on average become two).
__host__ __device__ __forceinline__ constexpr int col_es(int ns, int bx, int tsize) {
  return ns * bx + (ns != 6 ? 0
                    : tsize == 4 ? (bx == 1 ? 1 : bx == 2 ? 7 : bx == 4 ? 4 : 8)
                                 : (bx == 1 ? 5 : bx == 2 ? 2 : bx == 4 ? 4 : 0));
}

template <typename T>
struct ColGeo {
  int N;          // axis length
  long long est;  // global stride between consecutive axis elements
  long long base; // global offset of element 0 of column kx0 (component 0)
  int kx0;
  int outer;      // the other column axis' index (a frequency index after its forward pass)
};

template <typename T>
__device__ __forceinline__ ColGeo<T> col_geo(const Desc<T>& D, int axis, int BX, int blk) {
  ColGeo<T> g;
  const int ntx = (D.nh + BX - 1) / BX;
  const int tile = blk % ntx;
  const int o = blk / ntx;
  g.kx0 = tile * BX;
  g.outer = o;
  if (axis == 1) {
    g.N = D.n2;
    g.est = D.pitch;
    g.base = (long long)o * D.n2 * D.pitch + g.kx0;
  } else {
    g.N = D.n3;
    g.est = (long long)D.n2 * D.pitch;
    g.base = (long long)o * D.pitch + g.kx0;
  }
  return g;
}

// Tile loads keep kLoadBatch independent global loads in flight per thread.
constexpr int kLoadBatch = 8;

template <typename T, int BX, int ES>
__device__ __forceinline__ void col_load(const Desc<T>& D, const ColGeo<T>& g, int comp, cplx<T>* tl, int slot) {
  const cplx<T>* src = D.spec + (long long)comp * D.Vh + g.base;
  const int tot = g.N * BX;
  const int nthr = blockDim.x;
  for (int e0 = threadIdx.x; e0 < tot; e0 += nthr * kLoadBatch) {
    cplx<T> v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * nthr;
      const int y = e / BX, b = e % BX;
      v[u] = (e < tot && g.kx0 + b < D.nh) ? src[(long long)y * g.est + b] : cmake<T>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * nthr;
      const int y = e / BX, b = e % BX;
      if (e < tot) tl[y * ES + slot * BX + b] = v[u];
    }
  }
}

// Components 0..NC-1 into slots 0..NC-1 in one batched loop (more loads in flight).
template <typename T, int BX, int ES, int NC>
__device__ __forceinline__ void col_load_all(const Desc<T>& D, const ColGeo<T>& g, cplx<T>* tl) {
  const int per = g.N * BX;
  const int tot = NC * per;
  const int nthr = blockDim.x;
  for (int e0 = threadIdx.x; e0 < tot; e0 += nthr * kLoadBatch) {
    cplx<T> v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * nthr;
      const int comp = e / per, r = e - comp * per;
      const int y = r / BX, b = r % BX;
      v[u] = (e < tot && g.kx0 + b < D.nh) ? D.spec[(long long)comp * D.Vh + g.base + (long long)y * g.est + b]
                                            : cmake<T>(0, 0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * nthr;
      const int comp = e / per, r = e - comp * per;
      const int y = r / BX, b = r % BX;
      if (e < tot) tl[y * ES + comp * BX + b] = v[u];
    }
  }
}

template <typename T, int BX, int ES>
__device__ __forceinline__ void col_store(const Desc<T>& D, const ColGeo<T>& g, int comp, const cplx<T>* tl,
                                          int slot) {
  cplx<T>* dst = D.spec + (long long)comp * D.Vh + g.base;
  for (int e = threadIdx.x; e < g.N * BX; e += blockDim.x) {
    const int y = e / BX, b = e % BX;
    if (g.kx0 + b < D.nh) dst[(long long)y * g.est + b] = tl[y * ES + slot * BX + b];
  }
}

// frequency vector of tile element (axis index y, column b), in T
template <typename T>
__device__ __forceinline__ void col_xi(const Desc<T>& D, const ColGeo<T>& g, int axis, int y, int b, T& x1, T& x2,
                                       T& x3) {
  x1 = xi_of<T>(g.kx0 + b, D.n1, D.ks[0]);
  if (axis == 2) {
    x2 = xi_of<T>(g.outer, D.n2, D.ks[1]);
    x3 = xi_of<T>(y, D.n3, D.ks[2]);
  } else {
    x2 = xi_of<T>(y, D.n2, D.ks[1]);
    x3 = xi_of<T>(g.outer, D.n3, D.ks[2]);
  }
}

// Plain transform of one component (blockIdx.y) along `axis`.
template <typename T, int OP, int BX, int BATCH>
__global__ void __launch_bounds__(kColThreadsPlain, sizeof(T) == 8 ? 2 : 4)
    k_colplain(const Desc<T>* __restrict__ dd, BatchArgs<T> ba, int axis) {
  int blk;
  const Desc<T>* __restrict__ Dp = pick_ptr<T, BATCH>(dd, ba, blk);
  const Desc<T>& D = *Dp;
  if (D.sc->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const ColGeo<T> g = col_geo<T>(D, axis, BX, blk);
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* tl = tw + g.N;
  load_twiddles<T>(tw, D.tw[axis], g.N);
  const AxisPlan pl = D.ax[axis];
  const int comp = blockIdx.y;
  col_load<T, BX, BX>(D, g, comp, tl, 0);
  __syncthreads();
  fft_lines<T, BX, BX>(tl, pl, BX, 1, tw, OP == OP_FWD ? -1 : +1);
  col_store<T, BX, BX>(D, g, comp, tl, 0);
}

// Fused column pass along the axis hosting the spectral multiply; NS slots.
//   OP_GRAD: c inputs u^ -> s engineering strains e^ = (i/V) B(xi) u^
//   OP_DIV : s stresses sig^ -> c tractions t^ = (-theta/V) i B(xi)^T sig^
//   OP_PREC: c residuals r^ -> z^ = (1/V) (theta K(xi) + rho_bar I)^-1 r^, with the
//            Parseval partial sum of (r, z) over the half spectrum
// R16: the axis' schedule is pure radix 16 (only that stage kind is compiled in).
template <typename T, int OP, int BX, int NS, int BATCH, bool R16 = false>
__global__ void __launch_bounds__(kColThreadsOp, sizeof(T) == 8 ? 2 : 4)
    k_colop(const Desc<T>* __restrict__ dd, BatchArgs<T> ba, int axis) {
  constexpr int ES = col_es(NS, BX, (int)sizeof(T));
  int blk;
  const Desc<T>* __restrict__ Dp = pick_ptr<T, BATCH>(dd, ba, blk);
  const Desc<T>& D = *Dp;
  Scalars* sc = D.sc;
  if (sc->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const ColGeo<T> g = col_geo<T>(D, axis, BX, blk);
  const int N = g.N;
  cplx<T>* tw = reinterpret_cast<cplx<T>*>(smraw);
  cplx<T>* tl = tw + N;
  load_twiddles<T>(tw, D.tw[axis], N);
  const AxisPlan pl = D.ax[axis];
  // component counts, compile-time from the slot count: 3-D has NS = 6 (gradient,
  // divergence) or 3 (preconditioner), 2-D has 3 or 2
  constexpr int kC = (OP == OP_PREC) ? NS : (NS == 6 ? 3 : 2);
  constexpr int kS = (OP == OP_PREC) ? 0 : NS;
  constexpr int NIN = (OP == OP_DIV) ? kS : kC;
  constexpr int NOUT = (OP == OP_GRAD) ? kS : kC;
  // 3-D gradient / divergence: the six-slot side is transformed as two batches of three
  // slots, so a tile of BX columns needs only 3 BX N elements per batch in registers
  constexpr bool kSplit = OP != OP_PREC && NS == 6;
  col_load_all<T, BX, ES, NIN>(D, g, tl);
  __syncthreads();
  if (kSplit && NIN == 6) {
    fft_lines<T, ES, 3 * BX, R16>(tl, pl, 3 * BX, 1, tw, -1);
    fft_lines<T, ES, 3 * BX, R16>(tl + 3 * BX, pl, 3 * BX, 1, tw, -1);
  } else {
    fft_lines<T, ES, NIN * BX, R16>(tl, pl, NIN * BX, 1, tw, -1);
  }
  DotAcc<T> acc;
  for (int e = threadIdx.x; e < N * BX; e += blockDim.x) {
    const int y = e / BX, b = e % BX;
    cplx<T>* el = tl + y * ES + b;  // slot t at el[t * BX]
    T x1, x2, x3;
    col_xi<T>(D, g, axis, y, b, x1, x2, x3);
    if (OP == OP_GRAD) {
      const T iv = D.invV;
      if (kC == 3) {
        const cplx<T> u1 = el[0], u2 = el[BX], u3 = el[2 * BX];
        el[0] = cmuli<T>(cscale<T>(u1, x1 * iv), +1);
        el[BX] = cmuli<T>(cscale<T>(u2, x2 * iv), +1);
        el[2 * BX] = cmuli<T>(cscale<T>(u3, x3 * iv), +1);
        el[3 * BX] = cmuli<T>(cscale<T>(cadd<T>(cscale<T>(u3, x2), cscale<T>(u2, x3)), iv), +1);  // gamma_23
        el[4 * BX] = cmuli<T>(cscale<T>(cadd<T>(cscale<T>(u3, x1), cscale<T>(u1, x3)), iv), +1);  // gamma_13
        el[5 * BX] = cmuli<T>(cscale<T>(cadd<T>(cscale<T>(u2, x1), cscale<T>(u1, x2)), iv), +1);  // gamma_12
      } else {
        const cplx<T> u1 = el[0], u2 = el[BX];
        el[0] = cmuli<T>(cscale<T>(u1, x1 * iv), +1);
        el[BX] = cmuli<T>(cscale<T>(u2, x2 * iv), +1);
        el[2 * BX] = cmuli<T>(cscale<T>(cadd<T>(cscale<T>(u2, x1), cscale<T>(u1, x2)), iv), +1);  // gamma_12
      }
    } else if (OP == OP_DIV) {
      const T f = D.mthetaInvV;
      if (kC == 3) {
        const cplx<T> s11 = el[0], s22 = el[BX], s33 = el[2 * BX], s23 = el[3 * BX], s13 = el[4 * BX],
                      s12 = el[5 * BX];
        const cplx<T> t1 = cadd<T>(cadd<T>(cscale<T>(s11, x1), cscale<T>(s12, x2)), cscale<T>(s13, x3));
        const cplx<T> t2 = cadd<T>(cadd<T>(cscale<T>(s12, x1), cscale<T>(s22, x2)), cscale<T>(s23, x3));
        const cplx<T> t3 = cadd<T>(cadd<T>(cscale<T>(s13, x1), cscale<T>(s23, x2)), cscale<T>(s33, x3));
        el[0] = cmuli<T>(cscale<T>(t1, f), +1);
        el[BX] = cmuli<T>(cscale<T>(t2, f), +1);
        el[2 * BX] = cmuli<T>(cscale<T>(t3, f), +1);
      } else {
        const cplx<T> s11 = el[0], s22 = el[BX], s12 = el[2 * BX];
        const cplx<T> t1 = cadd<T>(cscale<T>(s11, x1), cscale<T>(s12, x2));
        const cplx<T> t2 = cadd<T>(cscale<T>(s12, x1), cscale<T>(s22, x2));
        el[0] = cmuli<T>(cscale<T>(t1, f), +1);
        el[BX] = cmuli<T>(cscale<T>(t2, f), +1);
      }
    } else {  // OP_PREC
      const int kx = g.kx0 + b;
      const T wgt = (kx >= D.nh) ? (T)0 : ((kx == 0 || 2 * kx == D.n1) ? (T)1 : (T)2);
      const T m0 = x1 * x1, m1 = x2 * x2, m2 = x3 * x3, m3 = x2 * x3, m4 = x1 * x3, m5 = x1 * x2;
      T Mv[6];
#pragma unroll
      for (int pr = 0; pr < 6; ++pr)
        Mv[pr] = D.kq[pr][0] * m0 + D.kq[pr][1] * m1 + D.kq[pr][2] * m2 + D.kq[pr][3] * m3 + D.kq[pr][4] * m4 +
                 D.kq[pr][5] * m5;
      Mv[0] += D.rhobar;
      Mv[1] += D.rhobar;
      Mv[2] += D.rhobar;
      const T iv = D.invV;
      if (kC == 3) {
        const T a = Mv[0], bb = Mv[1], cc = Mv[2], f = Mv[3], ee = Mv[4], d = Mv[5];
        const T A00 = bb * cc - f * f, A11 = a * cc - ee * ee, A22 = a * bb - d * d;
        const T A01 = ee * f - d * cc, A02 = d * f - bb * ee, A12 = d * ee - a * f;
        const T det = a * A00 + d * A01 + ee * A02;
        const T id = iv / det;
        const cplx<T> r1 = el[0], r2 = el[BX], r3 = el[2 * BX];
        const cplx<T> z1 = cscale<T>(cadd<T>(cadd<T>(cscale<T>(r1, A00), cscale<T>(r2, A01)), cscale<T>(r3, A02)), id);
        const cplx<T> z2 = cscale<T>(cadd<T>(cadd<T>(cscale<T>(r1, A01), cscale<T>(r2, A11)), cscale<T>(r3, A12)), id);
        const cplx<T> z3 = cscale<T>(cadd<T>(cadd<T>(cscale<T>(r1, A02), cscale<T>(r2, A12)), cscale<T>(r3, A22)), id);
        acc.add_prod(wgt * r1.x, z1.x);
        acc.add_prod(wgt * r1.y, z1.y);
        acc.add_prod(wgt * r2.x, z2.x);
        acc.add_prod(wgt * r2.y, z2.y);
        acc.add_prod(wgt * r3.x, z3.x);
        acc.add_prod(wgt * r3.y, z3.y);
        el[0] = z1;
        el[BX] = z2;
        el[2 * BX] = z3;
      } else {
        const T a = Mv[0], bb = Mv[1], d = Mv[5];
        const T id = iv / (a * bb - d * d);
        const cplx<T> r1 = el[0], r2 = el[BX];
        const cplx<T> z1 = cscale<T>(csub<T>(cscale<T>(r1, bb), cscale<T>(r2, d)), id);
        const cplx<T> z2 = cscale<T>(csub<T>(cscale<T>(r2, a), cscale<T>(r1, d)), id);
        acc.add_prod(wgt * r1.x, z1.x);
        acc.add_prod(wgt * r1.y, z1.y);
        acc.add_prod(wgt * r2.x, z2.x);
        acc.add_prod(wgt * r2.y, z2.y);
        el[0] = z1;
        el[BX] = z2;
      }
    }
  }
  if (OP == OP_PREC) {
    const double s = block_sum(acc.value());  // contains barriers
    if (threadIdx.x == 0) D.part[PT_B][blk] = s;
  }
  __syncthreads();
  if (kSplit && NOUT == 6) {
    fft_lines<T, ES, 3 * BX, R16>(tl, pl, 3 * BX, 1, tw, +1);
    fft_lines<T, ES, 3 * BX, R16>(tl + 3 * BX, pl, 3 * BX, 1, tw, +1);
  } else {
    fft_lines<T, ES, NOUT * BX, R16>(tl, pl, NOUT * BX, 1, tw, +1);
  }
  for (int k = 0; k < NOUT; ++k) col_store<T, BX, ES>(D, g, k, tl, k);
}

}  // namespace wfft
