// Batched mixed-radix FFT of lines held in shared memory.
//
// The DFT of Sec. 2.1.3 (Eq. Fourier_derivatives, Eq. frequencies) is
// computed by a self-sorting (Stockham) sequence of radix-R stages,
// R in {2,3,4,5,7,8}: with Ns the product of the radices already applied and
// n = N/R butterflies per line, butterfly j reads x[j + r n] (r < R),
// multiplies by W_{Ns R}^{(j mod Ns) r}, takes an R-point DFT and writes
// y[(j div Ns) Ns R + (j mod Ns) + r Ns].  Each thread keeps its butterflies'
// inputs in registers between two barriers, so every stage runs in place
// on one shared-memory buffer.  Output is in natural order.  Twiddles come
// from a per-stage table of W_{Ns R}^{r k} (host-built; conjugated for the
// inverse), so no trigonometric function is evaluated on the device.
#pragma once
#include "common.cuh"

namespace wfft {

// Butterflies a thread holds per stage for radix R: up to 16 complex values (14 and 15
// for radices 7, 3 and 5) in both precisions.  A stage transforms at most NbOf * threads
// butterflies, so the host accepts only plans whose every tile satisfies
// ceil(elements / R) <= NbOf * threads for each radix of its axis; with 256 threads a
// tile of three line pairs holds axes of up to 1194-1365 points.  Iterations past a
// tile's butterflies are predicated off, so small tiles pay only their index arithmetic.
template <typename T, int R> struct NbOf {
  static constexpr int v = (16 / R) > 0 ? 16 / R : 1;
};

// Radix-5 constants: cos(2 pi/5) = (sqrt5 - 1)/4, cos(4 pi/5) = -(sqrt5 + 1)/4,
// sin(2 pi/5), sin(4 pi/5).
#define WFFT_C51 0.30901699437494742410
#define WFFT_C52 (-0.80901699437494742410)
#define WFFT_S51 0.95105651629515357212
#define WFFT_S52 0.58778525229247312917
#define WFFT_S3 0.86602540378443864676   /* sin(pi/3) = sqrt3/2 */
#define WFFT_R2 0.70710678118654752440   /* 1/sqrt2 */
#define WFFT_C8 0.92387953251128675613   /* cos(pi/8) */
#define WFFT_S8 0.38268343236508977173   /* sin(pi/8) */

// In-register R-point DFT, X_q = sum_m v_m exp(sgn 2 pi i m q / R),
// sgn = -1 forward, +1 inverse.
template <typename T, int R>
struct Dft;

template <typename T>
struct Dft<T, 2> {
  __device__ __forceinline__ static void run(cplx<T>* v, int, const cplx<T>*, int) {
    cplx<T> a = v[0], b = v[1];
    v[0] = cadd<T>(a, b);
    v[1] = csub<T>(a, b);
  }
};

template <typename T>
struct Dft<T, 4> {
  __device__ __forceinline__ static void run(cplx<T>* v, int sgn, const cplx<T>*, int) {
    cplx<T> t0 = cadd<T>(v[0], v[2]), t1 = csub<T>(v[0], v[2]);
    cplx<T> t2 = cadd<T>(v[1], v[3]), t3 = cmuli<T>(csub<T>(v[1], v[3]), sgn);
    v[0] = cadd<T>(t0, t2);
    v[2] = csub<T>(t0, t2);
    v[1] = cadd<T>(t1, t3);
    v[3] = csub<T>(t1, t3);
  }
};

template <typename T>
struct Dft<T, 8> {
  __device__ __forceinline__ static void run(cplx<T>* v, int sgn, const cplx<T>*, int) {
    // even / odd radix-4 halves, then W_8^k combination
    cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4>::run(e, sgn, nullptr, 0);
    Dft<T, 4>::run(o, sgn, nullptr, 0);
    const T r2 = (T)WFFT_R2;
    // W_8^1 = (1 + sgn i)/sqrt2, W_8^2 = sgn i, W_8^3 = (-1 + sgn i)/sqrt2
    cplx<T> o1 = cscale<T>(cadd<T>(o[1], cmuli<T>(o[1], sgn)), r2);
    cplx<T> o2 = cmuli<T>(o[2], sgn);
    cplx<T> o3 = cscale<T>(csub<T>(cmuli<T>(o[3], sgn), o[3]), r2);
    v[0] = cadd<T>(e[0], o[0]);
    v[4] = csub<T>(e[0], o[0]);
    v[1] = cadd<T>(e[1], o1);
    v[5] = csub<T>(e[1], o1);
    v[2] = cadd<T>(e[2], o2);
    v[6] = csub<T>(e[2], o2);
    v[3] = cadd<T>(e[3], o3);
    v[7] = csub<T>(e[3], o3);
  }
};

// 16 = 4 x 4: X[k1 + 4 k2] = sum_n2 W16^(n2 k1) W4^(n2 k2) sum_n1 x[4 n1 + n2] W4^(n1 k1):
// four 4-point DFTs over n1, the twiddles W16^(n2 k1), four 4-point DFTs over n2.
template <typename T>
struct Dft<T, 16> {
  __device__ __forceinline__ static void run(cplx<T>* v, int sgn, const cplx<T>*, int) {
    cplx<T> y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[4 * n1 + n2];
      Dft<T, 4>::run(y[n2], sgn, nullptr, 0);
    }
    const T c8 = (T)WFFT_C8, s8 = (T)WFFT_S8, r2 = (T)WFFT_R2, sg = (T)sgn;
    // W16^m = (cos 2 pi m/16, sgn sin 2 pi m/16) for m = 1, 2, 3, 6, 9; W16^4 = sgn i
    const cplx<T> w1 = cmake<T>(c8, sg * s8), w2 = cmake<T>(r2, sg * r2), w3 = cmake<T>(s8, sg * c8);
    const cplx<T> w6 = cmake<T>(-r2, sg * r2), w9 = cmake<T>(-c8, -sg * s8);
    y[1][1] = cmul<T>(y[1][1], w1);
    y[1][2] = cmul<T>(y[1][2], w2);
    y[1][3] = cmul<T>(y[1][3], w3);
    y[2][1] = cmul<T>(y[2][1], w2);
    y[2][2] = cmuli<T>(y[2][2], sgn);
    y[2][3] = cmul<T>(y[2][3], w6);
    y[3][1] = cmul<T>(y[3][1], w3);
    y[3][2] = cmul<T>(y[3][2], w6);
    y[3][3] = cmul<T>(y[3][3], w9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      cplx<T> z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      Dft<T, 4>::run(z, sgn, nullptr, 0);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
    }
  }
};

template <typename T>
struct Dft<T, 3> {
  __device__ __forceinline__ static void run(cplx<T>* v, int sgn, const cplx<T>*, int) {
    cplx<T> s = cadd<T>(v[1], v[2]);
    cplx<T> d = cscale<T>(cmuli<T>(csub<T>(v[1], v[2]), sgn), (T)WFFT_S3);
    cplx<T> m = csub<T>(v[0], cscale<T>(s, (T)0.5));
    v[0] = cadd<T>(v[0], s);
    v[1] = cadd<T>(m, d);
    v[2] = csub<T>(m, d);
  }
};

template <typename T>
struct Dft<T, 5> {
  __device__ __forceinline__ static void run(cplx<T>* v, int sgn, const cplx<T>*, int) {
    cplx<T> b1 = cadd<T>(v[1], v[4]), b2 = cadd<T>(v[2], v[3]);
    cplx<T> d1 = csub<T>(v[1], v[4]), d2 = csub<T>(v[2], v[3]);
    const T c1 = (T)WFFT_C51, c2 = (T)WFFT_C52, s1 = (T)WFFT_S51, s2 = (T)WFFT_S52;
    cplx<T> a1 = cadd<T>(v[0], cadd<T>(cscale<T>(b1, c1), cscale<T>(b2, c2)));
    cplx<T> a2 = cadd<T>(v[0], cadd<T>(cscale<T>(b1, c2), cscale<T>(b2, c1)));
    cplx<T> q1 = cmuli<T>(cadd<T>(cscale<T>(d1, s1), cscale<T>(d2, s2)), sgn);
    cplx<T> q2 = cmuli<T>(csub<T>(cscale<T>(d1, s2), cscale<T>(d2, s1)), sgn);
    v[0] = cadd<T>(v[0], cadd<T>(b1, b2));
    v[1] = cadd<T>(a1, q1);
    v[4] = csub<T>(a1, q1);
    v[2] = cadd<T>(a2, q2);
    v[3] = csub<T>(a2, q2);
  }
};

// Radix 7: direct sum with the 7th roots of unity W_7^j = (cos 2 pi j/7, -sin 2 pi j/7),
// j = (m q) mod 7, conjugated for the inverse.
template <typename T>
struct Dft<T, 7> {
  __device__ __forceinline__ static void run(cplx<T>* v, int sgn, const cplx<T>*, int) {
    const T c7[7] = {(T)1, (T)0.62348980185873353053, (T)-0.22252093395631440429, (T)-0.90096886790241912624,
                     (T)-0.90096886790241912624, (T)-0.22252093395631440429, (T)0.62348980185873353053};
    const T s7[7] = {(T)0, (T)0.78183148246802980871, (T)0.97492791218182360702, (T)0.43388373911755812048,
                     (T)-0.43388373911755812048, (T)-0.97492791218182360702, (T)-0.78183148246802980871};
    cplx<T> in[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) in[m] = v[m];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      cplx<T> acc = in[0];
#pragma unroll
      for (int m = 1; m < 7; ++m) {
        const int j = (m * q) % 7;
        const cplx<T> w = cmake<T>(c7[j], sgn > 0 ? s7[j] : -s7[j]);
        acc = cadd<T>(acc, cmul<T>(in[m], w));
      }
      v[q] = acc;
    }
  }
};

// log2 of v if v is a power of two, else -1
__device__ __forceinline__ int log2_if_pow2(int v) { return (v & (v - 1)) ? -1 : __ffs(v) - 1; }

// Row tiles store element e of a line at rowpad(e): one unused slot after every
// 16 elements (128 bytes of FP32 complex).  The first stage of radix R writes
// butterfly outputs at stride R (R = 2, 4, 8, 16); with the pad, the 16 butterflies of
// a half-warp land in 16 distinct 8-byte bank pairs, and consecutive-element reads and
// writes of two lines of a warp (line stride N + N/16 + 1) take the minimum of two
// wavefronts (a one-slot pad per 8 elements made them take three).
__host__ __device__ __forceinline__ constexpr int rowpad(int e) { return e + (e >> 4); }
// Line stride (complex elements) of a row tile of lines of length N.
__host__ __device__ __forceinline__ constexpr int row_stride(int N) { return N + (N >> 4) + 1; }

// One in-place Stockham stage over `nlines` lines of length N.
// Row tiles (NL == 0, ES == 1): element e of line l at buf[l * lstride + rowpad(e)];
// consecutive threads take consecutive butterflies of a line.  Column tiles
// (NL > 0 lines and element stride ES, both compile-time): element e of line l at buf[l + e * ES];
// consecutive threads take consecutive lines.  Compile-time strides and line
// counts and shifts for power-of-two N and Ns keep the index arithmetic off the
// integer divider.
template <typename T, int R, int ES, int NL>
__device__ __forceinline__ void fft_stage(cplx<T>* buf, int N, int nlines, int lstride, int Ns, const cplx<T>* tw,
                                          int sgn) {
  constexpr int NB = NbOf<T, R>::v;
  constexpr bool LF = NL > 0;  // column tile (a 1-column tile has ES = 1)
  const int nb = N / R;
  const int nl = LF ? NL : nlines;
  const int total = nb * nl;
  const int nthr = blockDim.x;
  // read the thread index opaquely: keeps the compiler from hoisting every
  // stage's index arithmetic out of the callers' loops (register pressure)
  int tid;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
  const int lgnb = log2_if_pow2(nb);
  const int lgNs = log2_if_pow2(Ns);
  cplx<T> v[NB][R];
  int jj[NB], ll[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int id = tid + i * nthr;
    int line = 0, j = 0;
    if (LF) {
      line = id % NL;
      j = id / NL;
    } else if (lgnb >= 0) {
      j = id & (nb - 1);
      line = id >> lgnb;
    } else {
      j = id % nb;
      line = id / nb;
    }
    jj[i] = j;
    ll[i] = line;
    if (id < total) {
      const cplx<T>* src = LF ? buf + line : buf + (size_t)line * lstride;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = src[LF ? (j + r * nb) * ES : rowpad(j + r * nb)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int id = tid + i * nthr;
    if (id < total) {
      const int j = jj[i], line = ll[i];
      int k, g;
      if (lgNs >= 0) {
        k = j & (Ns - 1);
        g = j >> lgNs;
      } else {
        k = j % Ns;
        g = j / Ns;
      }
      if (Ns > 1) {
        // per-stage table: W_{Ns R}^{r k} at (Ns - 1) + (r - 1) Ns + k
        const cplx<T>* tws = tw + (Ns - 1) + k;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cplx<T> w = tws[(r - 1) * Ns];
          if (sgn > 0) w.y = -w.y;
          v[i][r] = cmul<T>(v[i][r], w);
        }
      }
      Dft<T, R>::run(v[i], sgn, tw, N);
      cplx<T>* dst = LF ? buf + line : buf + (size_t)line * lstride;
      const int base = g * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[LF ? (base + r * Ns) * ES : rowpad(base + r * Ns)] = v[i][r];
    }
  }
  __syncthreads();
}

// Elements a tile on an axis with a prime stage may hold per thread (the host accepts
// only tiles of at most kPrimeBatch * threads elements on such axes), and the output
// pairs (q, P - q) a thread then computes per prime stage: ceil(16 (P + 1) / (2 P)) = 9
// for P >= 11.
constexpr int kPrimeBatch = 16;
constexpr int kPrimeTasks = 9;
// a tile of kPrimeBatch * threads elements holds kPrimeBatch (P + 1) / (2 P) pairs per
// thread, largest for the smallest prime P = 11
static_assert(kPrimeTasks * 2 * 11 >= kPrimeBatch * (11 + 1), "prime-stage task batch too small for its tiles");

// General prime-length stage for the one prime factor P > 7 of an axis, run first
// (Ns = 1, no inter-stage twiddles): with n = N / P butterflies per line, output q of
// butterfly j is y[j P + q] = sum_r x[j + r n] W_P^{(r q) mod P} (conjugate roots for
// the inverse), a direct P-point DFT.  P is odd, so terms r and P - r share the root's
// cosine and negate its sine: with S_r = x_r + x_{P-r}, D_r = x_r - x_{P-r},
// A = sum_r S_r cos(2 pi r q / P) and B = sum_r i t_r D_r (t_r = -sin forward, +sin
// inverse), r = 1..(P-1)/2, the outputs q and P - q are x_0 + A + B and x_0 + A - B.
// One task computes such a pair from (P - 1) / 2 paired terms read from shared memory,
// the roots from the stage's table block (W_P^m at m - 1); a thread keeps up to
// kPrimeTasks pairs between the two barriers, so the stage runs in place like the
// others.  The loops over a thread's tasks are not unrolled: the pairs then live in
// local memory (L1) on this path only, and the stage takes no registers from the
// kernels it is compiled into (their other paths keep their register allocation).
// Cost: (P - 1) / 2 paired terms per two outputs, against about R products per
// radix-R element elsewhere: meant for the odd grid sizes of the paper (41, 43), not
// for speed.
template <typename T, int ES, int NL>
__device__ __forceinline__ void fft_stage_prime(cplx<T>* buf, int N, int P, int nlines, int lstride,
                                                const cplx<T>* tw, int sgn) {
  constexpr bool LF = NL > 0;
  const int nb = N / P;
  const int H = (P + 1) / 2;  // q = 0 .. (P - 1) / 2
  const int per_line = nb * H;
  const int tasks = per_line * (LF ? NL : nlines);
  const int nthr = blockDim.x;
  int tid;
  asm volatile("mov.u32 %0, %%tid.x;" : "=r"(tid));
  cplx<T> yq[kPrimeTasks], ym[kPrimeTasks];
#pragma unroll 1
  for (int i = 0; i < kPrimeTasks; ++i) {
    const int id = tid + i * nthr;
    if (id < tasks) {
      const int line = LF ? id % NL : id / per_line;
      const int t = LF ? id / NL : id - line * per_line;
      const int j = t / H, q = t - j * H;
      const cplx<T>* src = LF ? buf + line : buf + (size_t)line * lstride;
      const cplx<T> x0 = src[LF ? j * ES : rowpad(j)];
      cplx<T> A = cmake<T>((T)0, (T)0), B = cmake<T>((T)0, (T)0);
      int m = q;  // (r q) mod P for r = 1
      for (int r = 1; r <= (P - 1) / 2; ++r) {
        const cplx<T> a = src[LF ? (j + r * nb) * ES : rowpad(j + r * nb)];
        const cplx<T> b = src[LF ? (j + (P - r) * nb) * ES : rowpad(j + (P - r) * nb)];
        cplx<T> w = cmake<T>((T)1, (T)0);
        if (m) w = tw[m - 1];
        const T tr = sgn > 0 ? -w.y : w.y;
        const cplx<T> S = cadd<T>(a, b), D = csub<T>(a, b);
        A.x += S.x * w.x;
        A.y += S.y * w.x;
        B.x -= tr * D.y;
        B.y += tr * D.x;
        m += q;
        if (m >= P) m -= P;
      }
      const cplx<T> c = cadd<T>(x0, A);
      yq[i] = cadd<T>(c, B);
      ym[i] = csub<T>(c, B);
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int i = 0; i < kPrimeTasks; ++i) {
    const int id = tid + i * nthr;
    if (id < tasks) {
      const int line = LF ? id % NL : id / per_line;
      const int t = LF ? id / NL : id - line * per_line;
      const int j = t / H, q = t - j * H;
      cplx<T>* dst = LF ? buf + line : buf + (size_t)line * lstride;
      const int e = j * P + q;
      dst[LF ? e * ES : rowpad(e)] = yq[i];
      if (q) {
        const int e2 = j * P + P - q;
        dst[LF ? e2 * ES : rowpad(e2)] = ym[i];
      }
    }
  }
  __syncthreads();
}

// Full transform of `nlines` lines.  sgn = -1 forward, +1 inverse (unnormalised).
// Stages are applied radix by radix (the general prime stage, if the axis has a prime
// factor above 7, then 16s, 8s, 4s, 2s, 3s, 5s, 7s): the self-sorting
// formulation is valid for any order of the radices, and one loop per radix
// keeps each stage's registers apart.  ES = 1: row tiles with line stride
// `lstride` (nlines at run time), NL = 0; NL > 0: column tiles (line stride 1,
// element stride ES, NL lines).  Must be called by every thread of the block (barriers).
// ONLY16: the caller guarantees a pure radix-16 schedule (no prime stage either), and
// the other stage kinds are not compiled in (a smaller instruction footprint for
// kernels with several FFT calls).
template <typename T, int ES, int NL = 0, bool ONLY16 = false>
__device__ __forceinline__ void fft_lines(cplx<T>* buf, const AxisPlan& pl, int nlines, int lstride, const cplx<T>* tw,
                                          int sgn) {
  const int N = pl.n;
  int Ns = 1;
  if constexpr (!ONLY16) {
    if (pl.prime) {
      fft_stage_prime<T, ES, NL>(buf, N, pl.prime, nlines, lstride, tw, sgn);
      Ns = pl.prime;
    }
  }
  for (int s = 0; s < pl.cnt[6]; ++s, Ns *= 16) fft_stage<T, 16, ES, NL>(buf, N, nlines, lstride, Ns, tw, sgn);
  if constexpr (ONLY16) return;
  for (int s = 0; s < pl.cnt[0]; ++s, Ns *= 8) fft_stage<T, 8, ES, NL>(buf, N, nlines, lstride, Ns, tw, sgn);
  for (int s = 0; s < pl.cnt[1]; ++s, Ns *= 4) fft_stage<T, 4, ES, NL>(buf, N, nlines, lstride, Ns, tw, sgn);
  for (int s = 0; s < pl.cnt[2]; ++s, Ns *= 2) fft_stage<T, 2, ES, NL>(buf, N, nlines, lstride, Ns, tw, sgn);
  for (int s = 0; s < pl.cnt[3]; ++s, Ns *= 3) fft_stage<T, 3, ES, NL>(buf, N, nlines, lstride, Ns, tw, sgn);
  for (int s = 0; s < pl.cnt[4]; ++s, Ns *= 5) fft_stage<T, 5, ES, NL>(buf, N, nlines, lstride, Ns, tw, sgn);
  for (int s = 0; s < pl.cnt[5]; ++s, Ns *= 7) fft_stage<T, 7, ES, NL>(buf, N, nlines, lstride, Ns, tw, sgn);
}

}  // namespace wfft
