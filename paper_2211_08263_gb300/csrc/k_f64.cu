// FP64 instantiation of the pass kernels plus the FP64-only kernels of the
// Newmark step (Eq. Newmark, Eq. Fourier_ND_b, Alg. 2) and the single-block
// finalize kernels that turn block partial sums into the Krylov scalars.
#include <algorithm>
#include <cmath>

#include "finalize.cuh"
#include "passes_impl.cuh"
#include "profiler.cuh"

namespace wfft {

WFFT_INSTANTIATE(double)

// Predictor (Alg. 2 loop body, Eq. Fourier_ND_b):
//   u~ = u + dt v + dt^2 (1/2 - beta) a,  b = rho u~,
//   x0 = warm start with x0 = U(t_n) on the prescribed DOFs,
//   partial sums of || P b - sum_j U_j w_j ||^2 (w_j = P A(E e_j)).
// Blocks of an instance for its elementwise kernels (same rule as geo_blocks).
__device__ __forceinline__ int ew_blocks_dev(const Desc<double>& D) {
  const long long tot = (long long)D.c * D.V;
  long long nb = (tot + 255) / 256;
  if (nb > kEwBlocks) nb = kEwBlocks;
  return (int)(nb < 1 ? 1 : nb);
}

__global__ void __launch_bounds__(256) k_predict(const Desc<double>* __restrict__ dd, BatchArgs<double> ba) {
  int blk;
  const Desc<double>* __restrict__ Dp = pick_ptr<double, 1>(dd, ba, blk);
  const Desc<double>& D = *Dp;
  const int nblk = ew_blocks_dev(D);
  const Scalars* sc = D.sc;
  const long long V = D.V;
  const int c = D.c, nd = D.ndim;
  const double dt = D.dt, beta = D.beta;
  const double* u = reinterpret_cast<const double*>(D.slot[SL_U]);
  const double* v = reinterpret_cast<const double*>(D.slot[SL_V]);
  const double* a = reinterpret_cast<const double*>(D.slot[SL_A]);
  const double* w = reinterpret_cast<const double*>(D.slot[SL_W]);
  double* b = reinterpret_cast<double*>(D.slot[SL_B]);
  double* x = reinterpret_cast<double*>(D.slot[SL_X]);
  const double U0 = sc->Ug[0], U1 = sc->Ug[1], U2 = sc->Ug[2];
  const int warm = sc->warm;
  const bool use_au = sc->use_au != 0;
  const double dU0 = use_au ? sc->dU[0] : 0.0, dU1 = use_au ? sc->dU[1] : 0.0, dU2 = use_au ? sc->dU[2] : 0.0;
  const double* au = reinterpret_cast<const double*>(D.slot[SL_AU]);
  double* r64 = reinterpret_cast<double*>(D.slot[SL_R64]);
  double acc = 0.0, accr = 0.0;
  const long long tot = (long long)c * V;
  // component by component (no 64-bit division per element), voxels grid-strided
  const long long first = (long long)blk * blockDim.x + threadIdx.x, stride = (long long)nblk * blockDim.x;
  for (int k = 0; k < c; ++k)
  for (long long vox = first; vox < V; vox += stride) {
    const long long gi = (long long)k * V + vox;
    const double uu = u[gi], vv = v[gi], aa = a[gi];
    const double ut = uu + dt * vv + dt * dt * (0.5 - beta) * aa;
    const double bv = rho_at<double>(D, vox) * ut;
    double x0;
    if (warm == 1)
      x0 = uu + dt * vv + 0.5 * dt * dt * aa;
    else
      x0 = uu;  // increment warm starts add their FP32 increment after this pass
    const bool isg = (D.mask[vox] >> k) & 1;
    const double Uk = k == 0 ? U0 : (k == 1 ? U1 : U2);
    if (isg) x0 = Uk;
    b[gi] = bv;
    x[gi] = x0;
    // lifting field w_j enters only where U_j (or its increment) is nonzero: a zero
    // component's field is not read (the same result: 0 * w_j subtracts nothing)
    const double w0 = (U0 != 0.0 || dU0 != 0.0) ? w[gi] : 0.0;
    const double w1 = (nd > 1 && (U1 != 0.0 || dU1 != 0.0)) ? w[tot + gi] : 0.0;
    const double w2 = (nd > 2 && (U2 != 0.0 || dU2 != 0.0)) ? w[2 * tot + gi] : 0.0;
    if (!isg) {
      double t = bv - U0 * w0;
      if (nd > 1) t -= U1 * w1;
      if (nd > 2) t -= U2 * w2;
      acc += t * t;
    }
    if (use_au) {
      // x0 = u_{n-1} + sum_j dU_j E e_j, so P(b - A x0) = P(b - A u_{n-1}) - sum_j dU_j w_j,
      // with A u_{n-1} kept from the previous step's last FP64 residual evaluation
      double rv = bv - au[gi];
      rv -= dU0 * w0;
      if (nd > 1) rv -= dU1 * w1;
      if (nd > 2) rv -= dU2 * w2;
      if (isg) rv = 0.0;
      r64[gi] = rv;
      accr += rv * rv;
    }
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) D.part[PT_A][blk] = s;
  if (use_au) {
    const double sr = block_sum(accr);
    if (threadIdx.x == 0) D.part[PT_B][blk] = sr;
  }
}

// Corrector (Eq. Newmark): a_n = (u_n - u~)/(beta dt^2), v_n = v + dt((1-gamma) a + gamma a_n);
// partial sums of rho a_n per component (total force on the prescribed region), of rho |v_n|^2
// and of rho u_n . a_n (the energy of the step, see FIN_ENERGY's caller).
__global__ void __launch_bounds__(256) k_correct(const Desc<double>* __restrict__ dd, BatchArgs<double> ba) {
  int blk;
  const Desc<double>* __restrict__ Dp = pick_ptr<double, 1>(dd, ba, blk);
  const Desc<double>& D = *Dp;
  const int nblk = ew_blocks_dev(D);
  const Scalars* sc = D.sc;
  if (sc->status != 0) return;
  const long long V = D.V;
  const int c = D.c;
  const double dt = D.dt, beta = D.beta, gamma = D.gamma;
  // 1 / (beta dt^2) once: the per-element FP64 division (a reciprocal and Newton steps on
  // the FP64 pipe, the bound of this kernel) becomes one multiply
  const double inv_theta = 1.0 / (beta * dt * dt);
  double* u = reinterpret_cast<double*>(D.slot[SL_U]);
  double* v = reinterpret_cast<double*>(D.slot[SL_V]);
  double* a = reinterpret_cast<double*>(D.slot[SL_A]);
  const double* x = reinterpret_cast<const double*>(D.slot[SL_X]);
  const bool zf = sc->zero_free != 0;
  double acc[3] = {0.0, 0.0, 0.0};
  double ek = 0.0, eua = 0.0;
  // component by component (no 64-bit division per element), voxels grid-strided
  const long long first = (long long)blk * blockDim.x + threadIdx.x, stride = (long long)nblk * blockDim.x;
  for (int k = 0; k < c; ++k)
  for (long long vox = first; vox < V; vox += stride) {
    const long long gi = (long long)k * V + vox;
    const double uu = u[gi], vv = v[gi], aa = a[gi];
    const double ut = uu + dt * vv + dt * dt * (0.5 - beta) * aa;
    double xv = x[gi];
    if (zf && !((D.mask[vox] >> k) & 1)) xv = 0.0;
    const double an = (xv - ut) * inv_theta;
    const double vn = vv + dt * ((1.0 - gamma) * aa + gamma * an);
    u[gi] = xv;
    v[gi] = vn;
    a[gi] = an;
    const double rho = rho_at<double>(D, vox);
    const double f = rho * an;
    if (k == 0) acc[0] += f;
    else if (k == 1) acc[1] += f;
    else acc[2] += f;
    ek += rho * vn * vn;
    eua += xv * f;
  }
  for (int k = 0; k < 3; ++k) {
    const double s = block_sum(acc[k]);
    if (threadIdx.x == 0) D.part[k][blk] = s;
  }
  const double sk = block_sum(ek);
  if (threadIdx.x == 0) D.part[PT_D][blk] = sk;
  const double sua = block_sum(eua);
  if (threadIdx.x == 0) D.part[PT_E][blk] = sua;
}

// Unit lifting field E e_j: 1 on the prescribed DOFs of component j, 0 elsewhere.
__global__ void k_fill_unit(const Desc<double>* __restrict__ dd, int j, double* dst) {
  const Desc<double>& D = *dd;
  const long long V = D.V;
  const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x,
                  stride = (long long)gridDim.x * blockDim.x;
  for (int k = 0; k < D.c; ++k)
  for (long long vox = first; vox < V; vox += stride) {
    const long long gi = (long long)k * V + vox;
    dst[gi] = (k == j && ((D.mask[vox] >> k) & 1)) ? 1.0 : 0.0;
  }
}

// Explicit central-difference step (Sec. 2.3, Eq. Central_diff_rule), part 1:
// u_n = u + dt v + dt^2/2 a on every DOF.
__global__ void __launch_bounds__(256) k_explicit_predict(const Desc<double>* __restrict__ dd) {
  const Desc<double>& D = *dd;
  const long long tot = (long long)D.c * D.V;
  const double dt = D.dt;
  double* u = reinterpret_cast<double*>(D.slot[SL_U]);
  const double* v = reinterpret_cast<const double*>(D.slot[SL_V]);
  const double* a = reinterpret_cast<const double*>(D.slot[SL_A]);
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < tot;
       gi += (long long)gridDim.x * blockDim.x)
    u[gi] = u[gi] + dt * v[gi] + 0.5 * dt * dt * a[gi];
}

// Part 2 (Eq. Explicit_linear_momentum_arranged_3D), with q = -div(C : grad^s u_n)
// from the operator passes run at theta = 1:
//   v_b = v + dt/2 a + dt/(2 rho) div sigma,  f = 2 rho/dt (Udot - v_b) on Gamma (0 elsewhere),
//   v_n = v_b + dt/(2 rho) f,  a_n = 2 (v_n - v)/dt - a;
// partial sums of f per component (the force on Gamma).
__global__ void __launch_bounds__(256) k_explicit_update(const Desc<double>* __restrict__ dd, double U0, double U1,
                                                         double U2) {
  const Desc<double>& D = *dd;
  const long long V = D.V;
  const double dt = D.dt;
  double* v = reinterpret_cast<double*>(D.slot[SL_V]);
  double* a = reinterpret_cast<double*>(D.slot[SL_A]);
  const double* q = reinterpret_cast<const double*>(D.slot[SL_Q]);
  const double* un = reinterpret_cast<const double*>(D.slot[SL_U]);
  double acc[3] = {0.0, 0.0, 0.0};
  double ek = 0.0, euq = 0.0;
  const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x,
                  stride = (long long)gridDim.x * blockDim.x;
  for (int k = 0; k < D.c; ++k)
  for (long long vox = first; vox < V; vox += stride) {
    const long long gi = (long long)k * V + vox;
    const double rho = rho_at<double>(D, vox);
    const double vv = v[gi], aa = a[gi];
    const double vb = vv + 0.5 * dt * aa + dt / (2.0 * rho) * (-q[gi]);
    double vn = vb, f = 0.0;
    if ((D.mask[vox] >> k) & 1) {
      const double Uk = k == 0 ? U0 : (k == 1 ? U1 : U2);
      f = 2.0 * rho / dt * (Uk - vb);
      vn = vb + dt / (2.0 * rho) * f;
    }
    v[gi] = vn;
    a[gi] = 2.0 * (vn - vv) / dt - aa;
    if (k == 0) acc[0] += f;
    else if (k == 1) acc[1] += f;
    else acc[2] += f;
    ek += rho * vn * vn;
    euq += un[gi] * q[gi];
  }
  for (int k = 0; k < 3; ++k) {
    const double sum = block_sum(acc[k]);
    if (threadIdx.x == 0) D.part[k][blockIdx.x] = sum;
  }
  const double sk = block_sum(ek);
  if (threadIdx.x == 0) D.part[PT_D][blockIdx.x] = sk;
  const double suq = block_sum(euq);
  if (threadIdx.x == 0) D.part[PT_E][blockIdx.x] = suq;
}

// ---------------------------------------------------------------------------
// Green's-matrix treatment of Gamma (Sec. 2.2.3, Eqs. f_discrete, G, Vt,
// L-determination_ND; Alg. 2) -- small prescribed regions
// ---------------------------------------------------------------------------
// partial sums of ||f||^2 over a c-component field
__global__ void __launch_bounds__(256) k_green_norm2(const Desc<double>* __restrict__ dd, const double* f) {
  const Desc<double>& D = *dd;
  const long long tot = (long long)D.c * D.V;
  double acc = 0.0;
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < tot;
       gi += (long long)gridDim.x * blockDim.x)
    acc += f[gi] * f[gi];
  const double sum = block_sum(acc);
  if (threadIdx.x == 0) D.part[PT_A][blockIdx.x] = sum;
}

// out[i] = x[idx[i]] (column of G from one unit-force response, or u_b on Gamma)
__global__ void k_green_gather(const double* x, const long long* idx, long long n, double* out, long long stride) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i * stride] = x[idx[i]];
}

// V_i = U_k - ub[idx_i] with k the component of prescribed DOF i (Eq. Vt)
__global__ void k_green_mismatch(const double* ub, const long long* idx, long long n, long long V, double U0,
                                 double U1, double U2, double* out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(idx[i] / V);
    out[i] = (k == 0 ? U0 : (k == 1 ? U1 : U2)) - ub[idx[i]];
  }
}

// f = Ginv V: one warp per row (row-major n x n)
__global__ void k_green_gemv(const double* Ginv, const double* v, long long n, double* f) {
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  double acc = 0.0;
  for (long long j = lane; j < n; j += 32) acc += Ginv[row * n + j] * v[j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) f[row] = acc;
}

// b[idx_i] = f_i on a zeroed field
__global__ void k_green_scatter(double* b, const long long* idx, long long n, const double* f) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[idx[i]] = f[i];
}

// dst[idx] = 1 on a zeroed field (unit force of Eq. f_discrete)
__global__ void k_green_unit(double* b, long long gi) {
  if (blockIdx.x == 0 && threadIdx.x == 0) b[gi] = 1.0;
}

// x += y over a c-component field
__global__ void __launch_bounds__(256) k_green_axpy(double* x, const double* y, long long tot) {
  for (long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x; gi < tot;
       gi += (long long)gridDim.x * blockDim.x)
    x[gi] += y[gi];
}

// In-place Gauss-Jordan inversion of the SPD matrix G (no pivoting needed), pivot k:
//   piv = A_kk, col_i = A_ik;  A_kj <- (j == k ? 1 : A_kj) / piv;
//   A_ij <- (j == k ? 0 : A_ij) - col_i A_kj for i != k.
__global__ void k_gj_pivot(const double* A, long long n, long long k, double* col, double* piv) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    col[i] = A[i * n + k];
    if (i == k) *piv = A[k * n + k];
  }
}
__global__ void k_gj_row(double* A, long long n, long long k, const double* piv) {
  const double p = *piv;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
    A[k * n + j] = (j == k ? 1.0 : A[k * n + j]) / p;
}
__global__ void k_gj_eliminate(double* A, long long n, long long k, const double* col) {
  const long long tot = n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e - i * n;
    if (i == k) continue;
    A[e] = (j == k ? 0.0 : A[e]) - col[i] * A[k * n + j];
  }
}

static int ew_blocks(const Plan<double>& P) {
  const long long tot = (long long)P.h.c * P.h.V;
  long long nb = (tot + 255) / 256;
  if (nb > kEwBlocks) nb = kEwBlocks;
  return (int)(nb < 1 ? 1 : nb);
}

static BatchArgs<double> ew_args(const BatchLaunch<double>* bl) {
  BatchArgs<double> a;
  a.descs = bl ? bl->descs : nullptr;
  a.start = bl ? bl->start[GEO_EW] : nullptr;
  a.n = bl ? bl->n : 0;
  return a;
}
static double ew_cv(const Plan<double>& P, const BatchLaunch<double>* bl) {
  if (!bl) return (double)P.h.c * P.h.V;
  double s = 0;
  for (const Plan<double>* q : bl->plans) s += (double)q->h.c * q->h.V;
  return s;
}

void launch_predict(const Plan<double>& P, cudaStream_t st, const BatchLaunch<double>* bl) {
  const double cv = ew_cv(P, bl), mat = 3.0 * cv / P.h.c;
  const int nb = bl ? bl->total[GEO_EW] : ew_blocks(P);
  const BatchArgs<double> ba = ew_args(bl);
  prof_launch(0, KK_NEWMARK, 8 * cv * (3 + P.h.ndim + 2) + mat, cv * (8 + 2 * P.h.ndim), st,
              [&] { k_predict<<<nb, 256, 0, st>>>(P.d, ba); });
}
void launch_correct(const Plan<double>& P, cudaStream_t st, const BatchLaunch<double>* bl) {
  const double cv = ew_cv(P, bl), mat = 3.0 * cv / P.h.c;
  const int nb = bl ? bl->total[GEO_EW] : ew_blocks(P);
  const BatchArgs<double> ba = ew_args(bl);
  prof_launch(0, KK_NEWMARK, 8 * cv * 7 + mat, cv * 14, st, [&] { k_correct<<<nb, 256, 0, st>>>(P.d, ba); });
}
void launch_fill_unit(const Plan<double>& P, int j, double* dst, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 8.0 * P.h.c * P.h.V, 0.0, st, [&] { k_fill_unit<<<ew_blocks(P), 256, 0, st>>>(P.d, j, dst); });
}
int ew_block_count(const Plan<double>& P) { return ew_blocks(P); }
void launch_green_norm2(const Plan<double>& P, const double* f, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 8.0 * P.h.c * P.h.V, 2.0 * P.h.c * P.h.V, st,
              [&] { k_green_norm2<<<ew_blocks(P), 256, 0, st>>>(P.d, f); });
}
static int small_blocks(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 1024)); }
void launch_green_gather(const double* x, const long long* idx, long long n, double* out, long long stride,
                         cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 16.0 * n, 0.0, st,
              [&] { k_green_gather<<<small_blocks(n), 256, 0, st>>>(x, idx, n, out, stride); });
}
void launch_green_mismatch(const double* ub, const long long* idx, long long n, long long V, const double U[3],
                           double* out, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 24.0 * n, (double)n, st, [&] {
    k_green_mismatch<<<small_blocks(n), 256, 0, st>>>(ub, idx, n, V, U[0], U[1], U[2], out);
  });
}
void launch_green_gemv(const double* Ginv, const double* v, long long n, double* f, cudaStream_t st) {
  const long long warps = n, blocks = (warps * 32 + 255) / 256;
  prof_launch(0, KK_SCALAR, 8.0 * n * n, 2.0 * n * n, st,
              [&] { k_green_gemv<<<(int)blocks, 256, 0, st>>>(Ginv, v, n, f); });
}
void launch_green_scatter(double* b, const long long* idx, long long n, const double* f, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 24.0 * n, 0.0, st, [&] { k_green_scatter<<<small_blocks(n), 256, 0, st>>>(b, idx, n, f); });
}
void launch_green_unit(double* b, long long gi, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 8.0, 0.0, st, [&] { k_green_unit<<<1, 32, 0, st>>>(b, gi); });
}
void launch_green_axpy(const Plan<double>& P, double* x, const double* y, cudaStream_t st) {
  const long long tot = (long long)P.h.c * P.h.V;
  prof_launch(0, KK_NEWMARK, 24.0 * tot, (double)tot, st, [&] { k_green_axpy<<<ew_blocks(P), 256, 0, st>>>(x, y, tot); });
}
void launch_green_invert(double* A, long long n, double* col, double* piv, cudaStream_t st) {
  const int eb = (int)std::max<long long>(1, std::min<long long>((n * n + 255) / 256, 4096));
  for (long long k = 0; k < n; ++k) {
    prof_launch(0, KK_SCALAR, 8.0 * n, 0.0, st, [&] { k_gj_pivot<<<small_blocks(n), 256, 0, st>>>(A, n, k, col, piv); });
    prof_launch(0, KK_SCALAR, 16.0 * n, (double)n, st, [&] { k_gj_row<<<small_blocks(n), 256, 0, st>>>(A, n, k, piv); });
    prof_launch(0, KK_SCALAR, 16.0 * n * n, 2.0 * n * n, st,
                [&] { k_gj_eliminate<<<eb, 256, 0, st>>>(A, n, k, col); });
  }
}
void launch_explicit_predict(const Plan<double>& P, cudaStream_t st) {
  const double cv = (double)P.h.c * P.h.V;
  prof_launch(0, KK_NEWMARK, 8 * cv * 4, cv * 5, st, [&] { k_explicit_predict<<<ew_blocks(P), 256, 0, st>>>(P.d); });
}
void launch_explicit_update(const Plan<double>& P, const double Udot[3], cudaStream_t st) {
  const double cv = (double)P.h.c * P.h.V;
  prof_launch(0, KK_NEWMARK, 8 * cv * 5 + 3.0 * cv / P.h.c, cv * 14, st, [&] {
    k_explicit_update<<<ew_blocks(P), 256, 0, st>>>(P.d, Udot[0], Udot[1], Udot[2]);
  });
}

// ---------------------------------------------------------------------------
// incremental residual of a mixed solve
// ---------------------------------------------------------------------------
// Partial sums of ||d||^2 over the FP32 correction: FP32 squares summed in FP32 per
// thread (a relative error far below the 1 % the rounding estimate needs), FP64 across.
// BatchArgs as for the predictor (n = 0: one instance).
__global__ void __launch_bounds__(256) k_dnorm2(const Desc<double>* __restrict__ dd, BatchArgs<double> ba) {
  int blk;
  const Desc<double>* __restrict__ Dp = pick_ptr<double, 1>(dd, ba, blk);
  const Desc<double>& D = *Dp;
  const int nblk = ew_blocks_dev(D);
  const float* d = reinterpret_cast<const float*>(D.slot[SL_D]);
  const long long tot = (long long)D.c * D.V;
  float acc = 0.f;
  for (long long gi = (long long)blk * blockDim.x + threadIdx.x; gi < tot; gi += (long long)nblk * blockDim.x)
    acc = fmaf(d[gi], d[gi], acc);
  const double s = block_sum((double)acc);
  if (threadIdx.x == 0) D.part[PT_C][blk] = s;
}

__global__ void k_incr_begin(Scalars* sc64, Scalars* sc32, double rb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  sc64->rbound = rb;
  sc32->done = 0;
  sc32->status = 0;
}

// Grouped form: src = sc64 pointers then sc32 pointers of n instances; unfinished
// instances get their rounding estimate rb[i] and their FP32 scalars re-opened.
__global__ void k_incr_begin_batch(Scalars* const* src, int n, const double* rb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || src[i]->done) return;
  src[i]->rbound = rb[i];
  src[n + i]->done = 0;
  src[n + i]->status = 0;
}

// x += xc d, A x += xc q32, r = [P](b - A x): the residual of x + xc d from the stored
// FP64 product A x and the FP32 product of the correction (the same fold of d into x
// as the x pass of a full FP64 residual evaluation).  q32s[i]: instance i's FP32
// product (grouped launches); q32: the single instance's.
__global__ void __launch_bounds__(256) k_resid_incr(const Desc<double>* __restrict__ dd, BatchArgs<double> ba,
                                                    const float* __restrict__ q32, const float* const* q32s,
                                                    int masked) {
  int blk = blockIdx.x;
  const Desc<double>* Dp = dd;
  if (ba.n > 0) {  // instance index by binary search over the block prefix sums (as pick_ptr)
    int lo = 0, hi = ba.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(ba.start + mid) <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    blk = blockIdx.x - __ldg(ba.start + lo);
    Dp = ba.descs[lo];
    q32 = q32s[lo];
  }
  const Desc<double>& D = *Dp;
  if (D.sc->done) return;
  const int nblk = ew_blocks_dev(D);
  const double xc = D.sc_inner->xcoef;
  const long long V = D.V;
  const float* d = reinterpret_cast<const float*>(D.slot[SL_D]);
  const double* b = reinterpret_cast<const double*>(D.slot[SL_B]);
  double* x = reinterpret_cast<double*>(D.slot[SL_X]);
  double* au = reinterpret_cast<double*>(D.slot[SL_AU]);
  double* r = reinterpret_cast<double*>(D.slot[SL_R64]);
  double acc = 0.0;
  // component by component (no 64-bit division per element), voxels grid-strided
  const long long first = (long long)blk * blockDim.x + threadIdx.x, stride = (long long)nblk * blockDim.x;
  for (int k = 0; k < D.c; ++k)
  for (long long vox = first; vox < V; vox += stride) {
    const long long gi = (long long)k * V + vox;
    x[gi] = x[gi] + xc * (double)d[gi];
    const double ax = au[gi] + xc * (double)q32[gi];
    au[gi] = ax;
    double rv = b[gi] - ax;
    if (masked && ((D.mask[vox] >> k) & 1)) rv = 0.0;
    r[gi] = rv;
    acc = fma(rv, rv, acc);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) D.part[PT_A][blk] = s;
}

void launch_dnorm2(const Plan<double>& P, cudaStream_t st, const BatchLaunch<double>* bl) {
  const double cv = ew_cv(P, bl);
  const int nb = bl ? bl->total[GEO_EW] : ew_blocks(P);
  const BatchArgs<double> ba = ew_args(bl);
  prof_launch(0, KK_NEWMARK, 4.0 * cv, 2.0 * cv, st, [&] { k_dnorm2<<<nb, 256, 0, st>>>(P.d, ba); });
}
void launch_incr_begin(Scalars* sc64, Scalars* sc32, double rb, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] { k_incr_begin<<<1, 32, 0, st>>>(sc64, sc32, rb); });
}
void launch_incr_begin_batch(Scalars* const* src, int n, const double* rb, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] { k_incr_begin_batch<<<(n + 63) / 64, 64, 0, st>>>(src, n, rb); });
}
void launch_resid_incr(const Plan<double>& P, const float* q32, int masked, cudaStream_t st,
                       const BatchLaunch<double>* bl, const float* const* q32s) {
  const double cv = ew_cv(P, bl);
  const int nb = bl ? bl->total[GEO_EW] : ew_blocks(P);
  const BatchArgs<double> ba = ew_args(bl);
  prof_launch(0, KK_NEWMARK, cv * (8 * 6 + 4 * 2) + cv / P.h.c, cv * 6, st,
              [&] { k_resid_incr<<<nb, 256, 0, st>>>(P.d, ba, q32, q32s, masked); });
}

// ---------------------------------------------------------------------------
// finalize kernels (one block)
// ---------------------------------------------------------------------------
__device__ double fixed_order_sum(const double* p, int n) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
  return block_sum(s);
}

__device__ void fin_body(Scalars* sc, const double* pa, int na, const double* pb, int nb, const double* pc, int nc,
                         int mode, Scalars* sc2) {
  const double sa = pa ? fixed_order_sum(pa, na) : 0.0;
  const double sb = pb ? fixed_order_sum(pb, nb) : 0.0;
  const double scc = pc ? fixed_order_sum(pc, nc) : 0.0;
  if (threadIdx.x != 0) return;
  if (mode == FIN_CLOSE) {  // a grouped solve ended on a host limit: unfinished instances fail
    if (!sc->done) {
      sc->status = 4;
      sc->done = 1;
    }
    return;
  }
  // a finished solve is frozen: only the setup / bookkeeping modes still run
  if (sc->done && mode != FIN_REF && mode != FIN_REACT && mode != FIN_ENERGY) return;
  switch (mode) {
    case FIN_REF:
      sc->ref2 = sa;
      if (!isfinite(sa)) {
        sc->status = 5;
        sc->done = 1;
      } else if (sa == 0.0) {
        sc->zero_free = 1;
        sc->converged = 1;
        sc->done = 1;
        sc->rr = 0.0;
      }
      break;
    case FIN_RES0:
      sc->rr = sa;
      if (!isfinite(sa)) {
        sc->status = 5;
        sc->done = 1;
      } else if (sa <= sc->tol2 * sc->ref2) {
        sc->converged = 1;
        sc->done = 1;
      }
      break;
    case FIN_RZ0:
      sc->rz = sb;
      sc->first = 1;
      if (!isfinite(sb) || !(sb > 0.0)) {
        sc->status = 5;
        sc->done = 1;
      }
      break;
    case FIN_ALPHA:
      sc->pq = sa;
      sc->iter += 1;
      if (!isfinite(sa) || !(sa > 0.0)) {
        sc->status = 5;
        sc->done = 1;
      } else {
        sc->alpha = sc->rz / sa;
      }
      break;
    case FIN_BETA:
      sc->rr = sa;
      if (!isfinite(sa) || !isfinite(sb)) {
        sc->status = 5;
        sc->done = 1;
      } else if (sa <= sc->tol2 * sc->ref2) {
        sc->converged = 1;
        sc->done = 1;
      } else if (sc->iter >= sc->maxit) {
        sc->status = 4;
        sc->done = 1;
      } else if (!(sb > 0.0)) {
        sc->status = 5;
        sc->done = 1;
      } else {
        sc->beta = sb / sc->rz;
        sc->rz = sb;
        sc->first = 0;
      }
      break;
    case FIN_OUTER: {
      sc->rr = sa;
      // an incremental residual counts as converged only with its rounding bound added
      const double rb = sc->rbound;
      sc->rbound = 0.0;
      const double nrb = sqrt(sa) + rb;
      if (!isfinite(sa)) {
        sc->status = 5;
        sc->done = 1;
        sc2->done = 1;
      } else if (nrb * nrb <= sc->tol2 * sc->ref2) {
        sc->converged = 1;
        sc->done = 1;
        sc2->done = 1;
      } else {
        const double nr = sqrt(sa);
        sc2->scale = 1.0 / nr;
        sc2->xcoef = nr;
        sc2->ref2 = 1.0;
        // the inner solve reduces its (normalised) residual by inner_tol, or stops once it is
        // below floor_fac * tol * ref: the last sweep need not overshoot the outer target
        const double base = sc2->tol2_base > 0.0 ? sc2->tol2_base : sc2->tol2;
        const double fl = sc->floor_fac * sqrt(sc->tol2 * sc->ref2) / nr;
        sc2->tol2 = fmax(base, fl * fl);
        sc2->iter = 0;
        sc2->done = 0;
        sc2->first = 1;
        sc2->status = 0;
        sc2->converged = 0;
        sc2->zero_free = 0;
      }
      break;
    }
    case FIN_DNORM:
      sc->dnorm2 = scc;
      break;
    case FIN_REACT:
      sc->react[0] = sa;
      sc->react[1] = sb;
      sc->react[2] = scc;
      break;
    case FIN_ENERGY:
      sc->ekin2 = sa;
      sc->esum = sb;
      break;
    default:
      break;
  }
}

__global__ void k_fin(Scalars* sc, const double* pa, int na, const double* pb, int nb, const double* pc, int nc,
                      int mode, Scalars* sc2) {
  fin_body(sc, pa, na, pb, nb, pc, nc, mode, sc2);
}

// One block per instance of a grouped solve.
__global__ void k_fin_batch(const FinJob* jobs, int mode) {
  const FinJob& j = jobs[blockIdx.x];
  fin_body(j.sc, j.pa, j.na, j.pb, j.nb, j.pc, j.nc, mode, j.sc2);
}

__global__ void k_begin(Scalars* sc, double U0, double U1, double U2, int warm, double tol2, int maxit, int use_au,
                        double d0, double d1, double d2, double flr, double rb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  sc->Ug[0] = U0;
  sc->Ug[1] = U1;
  sc->Ug[2] = U2;
  sc->warm = warm;
  sc->tol2 = tol2;
  sc->maxit = maxit;
  sc->done = 0;
  sc->status = 0;
  sc->iter = 0;
  sc->first = 1;
  sc->zero_free = 0;
  sc->converged = 0;
  sc->scale = 1.0;
  sc->xcoef = 1.0;
  sc->rr = 0.0;
  sc->rz = 0.0;
  sc->alpha = 0.0;
  sc->beta = 0.0;
  sc->use_au = use_au;
  sc->dU[0] = d0;
  sc->dU[1] = d1;
  sc->dU[2] = d2;
  sc->tol2_base = tol2;
  sc->floor_fac = flr;
  sc->rbound = rb;
  sc->dnorm2 = 0.0;
}

__global__ void k_begin_batch(const BeginJob* jobs, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BeginJob& j = jobs[i];
  Scalars* sc = j.sc;
  for (int k = 0; k < 3; ++k) {
    sc->Ug[k] = j.U[k];
    sc->dU[k] = j.dU[k];
  }
  sc->warm = j.warm;
  sc->tol2 = j.tol2;
  sc->tol2_base = j.tol2;
  sc->floor_fac = 0.0;
  sc->rbound = j.rb;
  sc->dnorm2 = 0.0;
  sc->maxit = j.maxit;
  sc->done = 0;
  sc->status = 0;
  sc->iter = 0;
  sc->first = 1;
  sc->zero_free = 0;
  sc->converged = 0;
  sc->scale = 1.0;
  sc->xcoef = 1.0;
  sc->rr = 0.0;
  sc->rz = 0.0;
  sc->alpha = 0.0;
  sc->beta = 0.0;
  sc->use_au = j.use_au;
}

__global__ void k_set_done(Scalars* sc, int done) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc->done = done;
}

void launch_fin(Scalars* sc, const double* pa, int na, const double* pb, int nb, const double* pc, int nc, int mode,
                Scalars* sc2, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 8.0 * (na + nb + nc), (double)(na + nb + nc), st,
              [&] { k_fin<<<1, 256, 0, st>>>(sc, pa, na, pb, nb, pc, nc, mode, sc2); });
}
void launch_begin(Scalars* sc, const double U[3], int warm, double tol2, int maxit, cudaStream_t st, int use_au,
                  const double* dU, double flr, double rb) {
  const double d0 = dU ? dU[0] : 0.0, d1 = dU ? dU[1] : 0.0, d2 = dU ? dU[2] : 0.0;
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] {
    k_begin<<<1, 32, 0, st>>>(sc, U[0], U[1], U[2], warm, tol2, maxit, use_au, d0, d1, d2, flr, rb);
  });
}
void launch_fin_batch(const FinJob* jobs, int n, int mode, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] { k_fin_batch<<<n, 256, 0, st>>>(jobs, mode); });
}
void launch_begin_batch(const BeginJob* jobs, int n, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] { k_begin_batch<<<(n + 63) / 64, 64, 0, st>>>(jobs, n); });
}

__global__ void k_gather_scalars(Scalars* const* src, Scalars* dst, int n) {
  const int words = (int)(sizeof(Scalars) / sizeof(int));
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * words; t += gridDim.x * blockDim.x) {
    const int i = t / words, w = t - i * words;
    reinterpret_cast<int*>(dst + i)[w] = reinterpret_cast<const int*>(src[i])[w];
  }
}
void launch_gather_scalars(Scalars* const* src, Scalars* dst, int n, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] { k_gather_scalars<<<8, 256, 0, st>>>(src, dst, n); });
}

// Copy of a solve's two scalar blocks into host-mapped memory by the SMs themselves:
// the read-back needs no copy engine, so it does not queue behind a large
// asynchronous state download on another stream.
__global__ void k_read_scalars(const Scalars* a, const Scalars* b, Scalars* dst) {
  const int words = (int)(sizeof(Scalars) / sizeof(int));
  for (int t = threadIdx.x; t < 2 * words; t += blockDim.x) {
    const int i = t / words, w = t - i * words;
    reinterpret_cast<int*>(dst + i)[w] = reinterpret_cast<const int*>(i ? b : a)[w];
  }
}
void launch_read_scalars(const Scalars* a, const Scalars* b, Scalars* dst, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] { k_read_scalars<<<1, 128, 0, st>>>(a, b, dst); });
}

void launch_set_done(Scalars* sc, int done, cudaStream_t st) {
  prof_launch(0, KK_SCALAR, 0.0, 0.0, st, [&] { k_set_done<<<1, 32, 0, st>>>(sc, done); });
}

}  // namespace wfft
