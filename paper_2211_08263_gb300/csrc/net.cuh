// Learned warm start (not part of the paper's method): a 4-layer periodic 3-D
// convolution network predicting the next step's displacement increment as the
// Krylov initial guess.  BF16 weights and activations, FP32 accumulation on the
// tensor cores (mma.sync m16n8k16), FP32 master parameters and Adam for
// training.  Kernels and host code live in k_net.cu.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>

#include "../../include/wfft.h"

namespace wfft {

constexpr int kNetLayers = 4;
constexpr int kNetIn = 16;       // input feature channels
constexpr int kNetOut = 3;       // predicted displacement components
constexpr int kNetOutPad = 16;   // output channels as computed (one MMA k-step for the input gradient)
constexpr int32_t kNetMagic = 0x314E4657;  // "WFN1"
constexpr int kNetVersion = 1;

// Model blob: this header (8 int32) followed by the FP32 parameters of the four
// layers, per layer W[27][cout][cin] (offset o = 9 (dz+1) + 3 (dy+1) + (dx+1))
// then b[cout].
struct NetHeader {
  int32_t magic, version, layers, cin, hidden, cout, cout_pad, reserved;
};

struct NetDims {
  int hidden = 0;
  int cin[kNetLayers] = {}, cout[kNetLayers] = {};
  size_t woff[kNetLayers] = {}, boff[kNetLayers] = {};  // element offsets into the parameter vector
  size_t nparam = 0;
};
bool net_dims(int hidden, NetDims* d);
size_t net_blob_bytes(int hidden);
// Validates a blob; on success fills d.  Returns an error text or nullptr.
const char* net_parse(const void* blob, size_t bytes, NetDims* d);

// Device copy of one network.
struct NetDev {
  NetDims d;
  float* theta = nullptr;         // FP32 parameters (nparam)
  __nv_bfloat16* wb = nullptr;    // BF16 weights, forward layout (nparam, bias slots unused)
  __nv_bfloat16* wt = nullptr;    // BF16 weights, input-gradient layout (training only)
  int device = -1;
};
int net_upload(const void* blob, size_t bytes, bool training, NetDev** out, std::string* err);
void net_free(NetDev* n);

// One learned (or Taylor) warm start on a grid: fields of the current state.
struct WarmArgs {
  int n1, n2, n3, c;
  long long V;
  const double* u;     // FP64 [c][V]
  const double* v;
  const double* a;
  const uint8_t* mask;     // per voxel: bit k set = component k prescribed
  const uint16_t* phase;   // null: per-voxel material rows
  const float* ctab;       // FP32 material rows
  int cstride;
  const float* rhotab;
  int nd_idx[3], sh_idx[3], of_idx[3];  // row entries of the stiffness features (-1: none)
  float inv_nd[3], inv_sh, inv_of, inv_rhobar;
  double dt, theta;
  double Ug[3];            // U(t_n) on Gamma
};

// Work buffers of the inference path, sized for one grid.
struct NetWork {
  long long V = 0;
  int hidden = 0;
  __nv_bfloat16* x = nullptr;    // [V][16]
  __nv_bfloat16* h0 = nullptr;   // [V][hidden]
  __nv_bfloat16* h1 = nullptr;
  double* part = nullptr;        // block partial sums of the scale reduction
  float* scale = nullptr;        // [2]: s, 1/s
};
int net_work_alloc(NetWork* w, long long V, int hidden);
void net_work_free(NetWork* w);

// Reads and clears the error word of the tensor-core convolutions (a bounded wait expired);
// synchronises the device.
bool net_conv_timed_out();

// delta[k][vox] = dt v + dt^2/2 a (+ s y, y = net(features), when n != null) on free DOFs, 0 on Gamma.
void net_warm(const NetDev* n, NetWork* w, const WarmArgs& a, float* delta, cudaStream_t st);

// Fields of a handle for the warm-start kernels (defined with the handle in capi.cu).
int handle_warm_args(wfft_handle* h, const double U[3], WarmArgs* a, cudaStream_t* st, int* device);

}  // namespace wfft
