// Forward 3x3x3 periodic convolution of the warm-start network on the 5th-generation
// tensor cores (tcgen05.mma, BF16 operands from shared memory, FP32 accumulators in
// tensor memory).  Included by k_net.cu (uses its ConvArgs and EPI_* epilogues).
//
// GEMM shape.  Output channels are few (32), voxels many: a voxel tile is the MMA's N
// dimension (N = 128 voxels = 8 along x by 16 along y of one z-plane) and the rows are
// (dz, output channel) pairs.  For one input plane p, the nine in-plane offsets (dx, dy)
// and the input channels form the reduction:
//     D_p[(dz, co), v] = sum_{dx,dy} sum_ci W[dz, dy, dx][co][ci] X[p, v + (dx, dy)][ci],
// so every MMA of a plane reads one shifted window of the same staged halo plane.  Input
// plane p contributes block dz to output plane p - dz; output plane z is therefore
//     y_z = D_{z-1}[dz = -1] + D_z[dz = 0] + D_{z+1}[dz = +1],
// summed in the epilogue from three accumulator buffers (four 128-column buffers rotate
// in tensor memory, so the MMAs of plane z + 2 run while output plane z - 1 is formed).
// Row layout: row (dz + 1) COUT + co of the M = 128 rows (96 carry work for COUT = 32, the
// rest are zero weights).  A warp reads only its own 32-lane quarter of tensor memory, so
// the epilogue moves each block to shared memory ([dz][voxel][channel], a voxel's row
// padded to COUT + 4 floats so that 16-byte reads of consecutive voxels spread over the
// banks) and every thread then sums the three blocks for its voxel and half of the
// channels, adds the bias and stores 16-byte vectors of the channels-last output.
//
// Operand layouts (K-major, no swizzle): a core matrix is 8 rows of 16 bytes (8 BF16).
//   A (weights): [offset (dx,dy)][K step of 16][chunk of 8][row group][8 rows][16 B];
//                chunk stride (K direction) = 128 * 16 bytes, row-group stride 128 bytes.
//   B (a halo plane of 10 x 18 voxels): [chunk of 8 channels][y][x][16 B]; for offset
//                (dx, dy) the window starts (dy * 10 + dx) * 16 bytes in, 8 consecutive x
//                voxels form a core matrix, the next y row is 160 bytes on (N-group
//                stride), the next chunk 2880 bytes on (K direction).
// Roles (one CTA per SM, 13 warps, every hand-off an mbarrier):
//   loaders (warps 8-11): input plane g of a work unit (an 8 x 16 column of ZC output
//     planes) into stage g % NST with cp.async, once the MMAs of plane g - NST have
//     completed; after issuing plane g a loader thread waits for its copies of plane g - 1,
//     takes the generic-to-async proxy fence and arrives on that stage's "full" barrier
//     (a fence on the MMA thread instead waited for the MMAs in flight, ~400 cycles a plane);
//   MMA issue (warp 12, one lane): the 9 KH MMAs of plane g into accumulator g % NDB once
//     the stage is full and the accumulator's three readers (outputs g, g - 1, g - 2) are
//     done; descriptors are base descriptors plus compile-time offsets, so one MMA is issued
//     every ~72 cycles, the tensor pipe's rate for M = N = 128, K = 16; tcgen05.commit to
//     the accumulator's "full" and the stage's "empty" barriers;
//   epilogue (warps 0-7): two groups of four warps (one per lane quarter) take alternate
//     output planes; output plane k once plane k + 2 is committed: tensor memory -> the
//     group's exchange buffer, arrivals on the three accumulators read, then every thread
//     sums the three blocks for its voxel, adds the bias and stores the result.
// What bounds it: shared-memory bandwidth.  Per input plane the MMAs read 8 KB each (A and B
// operands, 144 KB for 32 input channels), the exchange writes and reads 96 KB and the
// loads write 11.5 KB: ~250 KB, ~1950 cycles at 128 B per clock, against ~2200 measured.
// Every wait is bounded; an expired wait raises a shared abort flag that ends every role,
// the kernel records an error word, waits (bounded) for its last commit, frees its tensor
// memory and returns.
#pragma once

namespace tcconv {

constexpr int TX = 8, TY = 16;            // output tile of a plane (MMA N = 128)
constexpr int HX = TX + 2, HY = TY + 2;   // halo plane
constexpr int NV = TX * TY;
constexpr int ZC = 32;                    // output planes per work unit
constexpr int NST = 3;                    // input-plane stages
constexpr int NDB = 4;                    // accumulator buffers of 128 columns
constexpr int kThreads = 416;             // warps 0-7 epilogue, 8-11 loads, 12 MMA issue
constexpr int kEpiThreads = 256;
constexpr int kLoadWarp0 = 8, kLoadThreads = 128;
constexpr int kMmaWarp = 12;
constexpr int kChunkStride = HX * HY * 16;  // 2880 bytes
constexpr unsigned kWaitLimit = 1u << 24;

template <int CIN, int COUT>
struct Geo {
  static constexpr int KCH = CIN / 8;
  static constexpr int KH = CIN / 16;
  static constexpr int PLANE = KCH * kChunkStride;
  static constexpr int ROWB = 128 * 16;  // bytes per A chunk (128 rows)
  static constexpr int ABYTES = 9 * KH * 2 * ROWB;
  static constexpr int SROW = COUT + 4;  // epilogue exchange [dz][voxel][channel], row padded to
                                         // spread 16-byte reads of consecutive voxels over the banks
  static constexpr int SBYTES = 3 * NV * SROW * 4;
  static constexpr int OFF_A = 0;
  static constexpr int OFF_P = ABYTES;
  static constexpr int OFF_S = OFF_P + NST * PLANE;
  static constexpr int OFF_BAR = OFF_S + 2 * SBYTES;      // mbarriers: acc full / empty, stage full / empty
  static constexpr int OFF_TAB = OFF_BAR + 8 * (2 * NDB + 2 * NST);  // TMEM slot, abort flag
  static constexpr int USED = OFF_TAB + 24;
  // two exchange buffers (one per epilogue group); at least 116 KB: one CTA per SM (each
  // holds all 512 tensor-memory columns)
  static constexpr size_t SMEM = USED > 116 * 1024 ? (size_t)USED : (size_t)116 * 1024;
  static_assert(CIN == 16 || CIN == 32, "input channels");
  // descriptor address fields are in 16-byte units and must not carry past 14 bits
  static_assert(PLANE % 16 == 0 && ROWB % 16 == 0 && SMEM <= 227 * 1024, "shared-memory layout");
  static_assert(COUT == 16 || COUT == 32, "output channels");
};

__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  // D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), both K-major,
  // N >> 3 at bit 17, M >> 4 at bit 24
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t kstride, uint32_t nstride) {
  // no swizzle: start address, K-direction core-matrix stride (leading byte offset),
  // M/N-direction 8-row-group stride (stride byte offset), descriptor version 1
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((kstride >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((nstride >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t id, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; gives up early once another role has flagged an abort.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar, uint32_t count = 1) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar), "r"(count) : "memory");
}
// Named barrier `id` of one epilogue group (128 threads).
__device__ __forceinline__ void epi_sync(uint32_t id) { asm volatile("bar.sync %0, 128;\n" ::"r"(id) : "memory"); }
// true on every thread of the group iff pred holds on all 128 (barrier `id` with an AND reduction)
__device__ __forceinline__ bool epi_all(uint32_t id, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %2, 0;\nbar.red.and.pred q, %1, 128, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(id), "r"((uint32_t)pred)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 columns of the 32 lanes of this warp's quarter, starting at taddr (asynchronous:
// the registers are valid after tmem_wait()).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

}  // namespace tcconv

// Work unit u of a grid: tile (ux, uy) of 8 x 16 voxels, output planes [zc*ZC, zc*ZC + nz).
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(tcconv::kThreads, 1) k_conv_tc(ConvArgs p, int* err) {
  using G = tcconv::Geo<CIN, COUT>;
  constexpr int TX = tcconv::TX, TY = tcconv::TY, HX = tcconv::HX, HY = tcconv::HY, NV = tcconv::NV;
  constexpr int ZC = tcconv::ZC, NST = tcconv::NST, NDB = tcconv::NDB, kThreads = tcconv::kThreads;
  constexpr int kChunkStride = tcconv::kChunkStride;
  using namespace tcconv;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* As = sm + G::OFF_A;
  unsigned char* Ps = sm + G::OFF_P;
  float* S = reinterpret_cast<float*>(sm + G::OFF_S);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + G::OFF_BAR);
  uint64_t* acc_full = bars;
  uint64_t* acc_empty = bars + NDB;
  uint64_t* st_full = bars + 2 * NDB;
  uint64_t* st_empty = bars + 2 * NDB + NST;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + G::OFF_TAB);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + G::OFF_TAB + 4);
  volatile long long* last_issued = reinterpret_cast<volatile long long*>(sm + G::OFF_TAB + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights into the A layout: W[27][COUT][CIN] -> [o9][kh][ch][row group][8 rows][16 B]
  for (int id = tid; id < 27 * COUT * G::KCH; id += kThreads) {
    const int c8 = id % G::KCH, r = id / G::KCH;
    const int co = r % COUT, o = r / COUT;
    const int dzi = o / 9, o9 = o % 9;
    const int row = dzi * COUT + co, kh = c8 >> 1, ch = c8 & 1;
    const int off = ((o9 * G::KH + kh) * 2 + ch) * G::ROWB + (row >> 3) * 128 + (row & 7) * 16;
    cp16(smem_u32(As + off), p.W + (size_t)(o * COUT + co) * CIN + 8 * c8);
  }
  // rows past 3 COUT: zero weights (their accumulator lanes are never read)
  for (int id = tid; id < 9 * G::KH * 2 * 128; id += kThreads) {
    const int row = id & 127;
    if (row < 3 * COUT) continue;
    *reinterpret_cast<uint4*>(As + (id >> 7) * G::ROWB + (row >> 3) * 128 + (row & 7) * 16) = make_uint4(0, 0, 0, 0);
  }
  cp_commit();
  if (tid == 0) {
    for (int b = 0; b < NDB; ++b) {
      mbar_init(smem_u32(acc_full + b), 1);
      mbar_init(smem_u32(acc_empty + b), 3);  // the three outputs that read a plane's blocks
    }
    for (int b = 0; b < NST; ++b) {
      mbar_init(smem_u32(st_full + b), kLoadThreads);
      mbar_init(smem_u32(st_empty + b), 1);
    }
    *abort_flag = 0;
    *last_issued = -1;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  cp_wait_all();
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const int nux = p.n1 / TX, nuy = p.n2 / TY, nzc = (p.n3 + ZC - 1) / ZC;
  const long long units = (long long)nux * nuy * nzc;

  if (warp >= kLoadWarp0 && warp < kMmaWarp) {
    // ---- loads: input plane j of a unit into stage g % NST once the MMAs of plane g - NST are done.
    // A thread copies the same (chunk, halo voxel) slots of every plane of a unit: their
    // shared-memory offsets and in-plane global offsets are set once per unit.
    constexpr int NSLOT = HX * HY * G::KCH;
    constexpr int PER = (NSLOT + kLoadThreads - 1) / kLoadThreads;
    const int lt = tid - kLoadWarp0 * 32;
    long long gp = 0;
    long long pend = -1;  // plane whose copies are issued but not yet announced
    bool lok = true;
    for (long long u = blockIdx.x; u < units && lok; u += gridDim.x) {
      const int ux = (int)(u % nux);
      const long long r1 = u / nux;
      const int uy = (int)(r1 % nuy), zc = (int)(r1 / nuy);
      const int x0 = ux * TX, y0 = uy * TY, zb = zc * ZC;
      const int NP = min(ZC, p.n3 - zb) + 2;
      uint32_t soff[PER];
      long long goff[PER];
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int id = lt + i * kLoadThreads;
        soff[i] = 0;
        goff[i] = -1;
        if (id < NSLOT) {
          const int c8 = id % G::KCH, hv = id / G::KCH;
          const int hx = hv % HX, hy = hv / HX;
          int x = x0 - 1 + hx, y = y0 - 1 + hy;
          x += x < 0 ? p.n1 : (x >= p.n1 ? -p.n1 : 0);
          y += y < 0 ? p.n2 : (y >= p.n2 ? -p.n2 : 0);
          soff[i] = (uint32_t)(c8 * kChunkStride + (hy * HX + hx) * 16);
          goff[i] = ((long long)y * p.n1 + x) * CIN + 8 * c8;
        }
      }
      const long long plane_elems = (long long)p.n1 * p.n2 * CIN;
      for (int j = 0; j < NP; ++j) {
        const long long g = gp + j;
        const int st = (int)(g % NST);
        const bool ok = g < NST || mbar_wait(smem_u32(st_empty + st), (uint32_t)(((g - NST) / NST) & 1), abort_flag);
        if (!__all_sync(0xffffffffu, ok)) {
          lok = false;
          break;
        }
        const int z = wrapi(zb - 1 + j, p.n3);
        const uint32_t dst = smem_u32(Ps + (size_t)st * G::PLANE);
        const bf16* src = p.in + (long long)z * plane_elems;
#pragma unroll
        for (int i = 0; i < PER; ++i)
          if (goff[i] >= 0) cp16(dst + soff[i], src + goff[i]);
        cp_commit();
        // the previous plane's copies have landed (all groups but the newest): a proxy fence
        // makes them visible to the tensor cores' reads, then the stage is announced
        if (pend >= 0) {
          asm volatile("cp.async.wait_group 1;\n" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mbar_arrive(smem_u32(st_full + (int)(pend % NST)));
        }
        pend = g;
      }
      if (__any_sync(0xffffffffu, *abort_flag != 0)) lok = false;
      gp += NP;
    }
    if (lok && pend >= 0) {
      cp_wait_all();
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(smem_u32(st_full + (int)(pend % NST)));
    }
  } else if (warp == kMmaWarp) {
    // ---- MMAs of plane g into accumulator g % NDB (free once output g - NDB has read it);
    // the whole warp waits, lane 0 issues.  The descriptors of a plane's MMAs are the stage's
    // and the weights' base descriptors plus compile-time offsets (address field in 16-byte
    // units; every shared address is below 256 KB, so the 14-bit field never carries), so
    // the issue loop is a handful of instructions per MMA and keeps the tensor pipe fed.
    const uint32_t idesc = idesc_bf16_f32(128, NV);
    const uint64_t adesc = smem_desc(smem_u32(As), G::ROWB, 128);
    const uint64_t bdesc = smem_desc(smem_u32(Ps), kChunkStride, HX * 16);
    long long gp = 0;
    bool run = true;
    for (long long u = blockIdx.x; u < units && run; u += gridDim.x) {
      const long long r1 = u / nux;
      const int zc = (int)(r1 / nuy);
      const int NP = min(ZC, p.n3 - zc * ZC) + 2;
      for (int j = 0; j < NP; ++j) {
        const long long g = gp + j;
        const int st = (int)(g % NST), db = (int)(g % NDB);
        bool ok = mbar_wait(smem_u32(st_full + st), (uint32_t)((g / NST) & 1), abort_flag);
        ok = ok && (g < NDB || mbar_wait(smem_u32(acc_empty + db), (uint32_t)(((g - NDB) / NDB) & 1), abort_flag));
        if (!__all_sync(0xffffffffu, ok)) {
          run = false;
          break;
        }
        if (lane == 0) {
          // (the loaders took the proxy fence before announcing the stage)
          tc_fence_after();
          const uint64_t bd = bdesc + (uint64_t)((st * G::PLANE) >> 4);
          const uint32_t dt = tbase + (uint32_t)(db * NV);
#pragma unroll
          for (int o9 = 0; o9 < 9; ++o9) {
#pragma unroll
            for (int kh = 0; kh < G::KH; ++kh) {
              const uint32_t aoff = (uint32_t)(((o9 * G::KH + kh) * 2 * G::ROWB) >> 4);
              const uint32_t boff = (uint32_t)((((o9 / 3) * HX + o9 % 3) * 16 + kh * 2 * kChunkStride) >> 4);
              mma_f16(dt, adesc + aoff, bd + boff, idesc, (o9 | kh) ? 1 : 0);
            }
          }
          mma_commit(smem_u32(acc_full + db));
          mma_commit(smem_u32(st_empty + st));
          *last_issued = g;
        }
        __syncwarp();
      }
      gp += NP;
    }
  } else {
    // ---- epilogue (warps 0-7): two groups of four warps (warps 4G .. 4G + 3, one per lane
    // quarter) take alternate output planes of a unit (group G: k = G, G + 2, ...), each with
    // its own exchange buffer and named barrier, so that one group's exchange runs while the
    // other sums and stores.  Output plane k reads the blocks of the accumulators of planes
    // k, k + 1, k + 2, and an accumulator is free once its three readers (outputs j, j - 1,
    // j - 2) have read it: every output arrives on all three after its reads; at the ends of
    // a unit the first and last outputs arrive for the readers that do not exist.
    const int q = warp & 3, grp = warp >> 2, gt = tid & 127;
    const uint32_t barid = 1 + grp;
    float* Sg = S + (size_t)grp * (G::SBYTES / 4);
    constexpr int NB = EPI == EPI_RELU ? COUT : 4;
    float bias[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) bias[c] = p.bias[c];
    long long gp = 0;
    bool ok = true;
    for (long long u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int ux = (int)(u % nux);
      const long long r1 = u / nux;
      const int uy = (int)(r1 % nuy), zc = (int)(r1 / nuy);
      const int x0 = ux * TX, y0 = uy * TY, zb = zc * ZC;
      const int nz = min(ZC, p.n3 - zb);
      for (int k = grp; k < nz; k += 2) {
        const long long g = gp + k;
        ok = epi_all(barid, mbar_wait(smem_u32(acc_full + ((g + 2) % NDB)), (uint32_t)(((g + 2) / NDB) & 1), abort_flag));
        if (!ok) break;
        tc_fence_after();
        if (32 * q < 3 * COUT) {
          const int r = 32 * q + lane;
          const int b = r / COUT, co = r % COUT;
          const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16);
#pragma unroll 1
          for (int bb = (32 * q) / COUT; bb <= (32 * q + 31) / COUT && bb < 3; ++bb) {
            const uint32_t tb = tq + (uint32_t)(((g + bb) % NDB) * NV);
#pragma unroll 1
            for (int c0 = 0; c0 < NV; c0 += 64) {
              uint32_t v0[32], v1[32];
              tmem_ld32(tb + c0, v0);
              tmem_ld32(tb + c0 + 32, v1);
              tmem_wait();
              if (b == bb) {
                float* dst = Sg + (b * NV + c0) * G::SROW + co;
#pragma unroll
                for (int e = 0; e < 32; ++e) dst[e * G::SROW] = __uint_as_float(v0[e]);
#pragma unroll
                for (int e = 0; e < 32; ++e) dst[(32 + e) * G::SROW] = __uint_as_float(v1[e]);
              }
            }
          }
        }
        tc_fence_before();
        epi_sync(barid);
        if (gt == 0) {
          mbar_arrive(smem_u32(acc_empty + (g % NDB)), k == 0 ? 3u : 1u);
          mbar_arrive(smem_u32(acc_empty + ((g + 1) % NDB)), 1u + (k == 0) + (k == nz - 1));
          mbar_arrive(smem_u32(acc_empty + ((g + 2) % NDB)), k == nz - 1 ? 3u : 1u);
        }
        {
          const int v = gt;  // voxel of the tile
          const int x = x0 + (v & 7), y = y0 + (v >> 3), z = zb + k;
          const long long vox = ((long long)z * p.n2 + y) * p.n1 + x;
          const float* s0 = Sg + (0 * NV + v) * G::SROW;
          const float* s1 = Sg + (1 * NV + v) * G::SROW;
          const float* s2 = Sg + (2 * NV + v) * G::SROW;
          if (EPI == EPI_RELU) {
            uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(p.out) + vox * COUT);
#pragma unroll
            for (int c8 = 0; c8 < COUT; c8 += 8) {
              uint32_t pk[4];
#pragma unroll
              for (int cc = 0; cc < 8; cc += 4) {
                const int c = c8 + cc;
                const float4 a = *reinterpret_cast<const float4*>(s0 + c);
                const float4 b4 = *reinterpret_cast<const float4*>(s1 + c);
                const float4 d = *reinterpret_cast<const float4*>(s2 + c);
                const float y0v = fmaxf(a.x + b4.x + d.x + bias[c], 0.f), y1v = fmaxf(a.y + b4.y + d.y + bias[c + 1], 0.f);
                const float y2v = fmaxf(a.z + b4.z + d.z + bias[c + 2], 0.f), y3v = fmaxf(a.w + b4.w + d.w + bias[c + 3], 0.f);
                __nv_bfloat162 h0 = __floats2bfloat162_rn(y0v, y1v), h1 = __floats2bfloat162_rn(y2v, y3v);
                pk[cc >> 1] = *reinterpret_cast<uint32_t*>(&h0);
                pk[(cc >> 1) + 1] = *reinterpret_cast<uint32_t*>(&h1);
              }
              dst[c8 / 8] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
          } else if (EPI == EPI_LINEAR) {
            const float4 a = *reinterpret_cast<const float4*>(s0);
            const float4 b4 = *reinterpret_cast<const float4*>(s1);
            const float4 d = *reinterpret_cast<const float4*>(s2);
            reinterpret_cast<float4*>(p.out)[vox] =
                make_float4(a.x + b4.x + d.x + bias[0], a.y + b4.y + d.y + bias[1], a.z + b4.z + d.z + bias[2],
                            a.w + b4.w + d.w + bias[3]);
          } else {  // EPI_WARM: delta += s (y + b) on free DOFs
            const float s = p.scale[0];
            const uint8_t mk = p.mask ? p.mask[vox] : (uint8_t)0;
            float* delta = reinterpret_cast<float*>(p.out);
            const float4 a = *reinterpret_cast<const float4*>(s0);
            const float4 b4 = *reinterpret_cast<const float4*>(s1);
            const float4 d = *reinterpret_cast<const float4*>(s2);
            const float y3[3] = {a.x + b4.x + d.x + bias[0], a.y + b4.y + d.y + bias[1], a.z + b4.z + d.z + bias[2]};
            float d3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) d3[c] = c < p.c ? delta[(long long)c * p.V + vox] : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c)
              if (c < p.c && !((mk >> c) & 1)) delta[(long long)c * p.V + vox] = d3[c] + s * y3[c];
          }
        }
        epi_sync(barid);  // the group's exchange buffer is reused by its next output
      }
      gp += nz + 2;
    }
  }
  // drain: every role has left its loop; on an abort, wait (bounded) for the MMAs still
  // in flight before the tensor memory is freed
  __syncwarp();
  __syncthreads();
  if (*abort_flag) {
    if (tid == 0) atomicExch(err, 1);
    // the MMAs of the last committed plane (and so every earlier one), bounded
    const long long gl = *last_issued;
    if (warp == 0 && gl >= 0) {
      const uint32_t b = smem_u32(acc_full + (gl % NDB));
      for (unsigned it = 0; it < kWaitLimit && !mbar_try(b, (uint32_t)((gl / NDB) & 1)); ++it) {
      }
    }
  }
  cp_wait_all();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tbase));
}
