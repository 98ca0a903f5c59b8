// Host driver of the learned initial guess's network (mg_unet_* in mg.h): a
// 3D U-Net with BF16 weights and activations and FP32 accumulation, whose
// convolutions run on the tcgen05 kernel of kernels_unet.cu.
//
// Architecture (levels L, base channels c; level l has c_l = c 2^l channels
// and grid size n / 2^l):
//   down path, l = 0 .. L-1: input (level 0: the three feature channels,
//     padded to 16; level l > 0: the 2x2x2 mean of level l-1's output), then
//     two 3x3x3 convolutions (zero padding, bias) each followed by ReLU;
//   up path, l = L-2 .. 0: the level below's output upsampled by 2 (nearest)
//     and concatenated after level l's down output (skip first), then two
//     3x3x3 convolutions with ReLU;
//   head: a 1x1x1 convolution to one channel, times the active mask.
// The concatenation is one buffer per level: level l's second down
// convolution writes its channels [0, c_l) and the upsampling its channels
// [c_l, c_l + c_{l+1}), so no copy is made.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mg.h"
#include "mg_internal.h"
#include "unet_internal.h"

namespace gbmg {
void set_thread_error(const char* msg);        // mg_capi.cu
bool is_device_ptr(const void* p, int device);  // mg_capi.cu
}  // namespace gbmg

using namespace gbmg;

namespace {

constexpr int kMaxNetLevels = 6;

struct Tensor {
  __nv_bfloat16* p = nullptr;
  int stride = 0;  // channels per voxel of the buffer
  int off = 0;     // first channel of the tensor
  int c = 0;       // channels of the tensor
  int W = 0, H = 0, D = 0;
  long long voxels() const { return (long long)W * H * D; }
};

struct Conv {
  int cin = 0, cin_pad = 0, cout = 0, level = 0;
  long long off_w = 0, off_b = 0;  // offsets in the flat parameter (and gradient) arrays
  float* w = nullptr;   // FP32 master weights [cout][cin][27]
  float* b = nullptr;   // [cout]
  float* dw = nullptr;  // gradients, same layout
  float* db = nullptr;
  __nv_bfloat16* wf = nullptr;  // packed forward weights
  __nv_bfloat16* wb = nullptr;  // packed backward-data weights (null for the first convolution)
  Tensor in, out;
  CUtensorMap map_in;
  ConvArgs args;
  int grid = 0;
  size_t smem = 0;
  // backward
  Tensor gz;                 // gradient of the pre-activation, [V][cout]
  CUtensorMap map_gz_bd;     // gz as the backward-data convolution's input
  ConvArgs bargs;
  int bgrid = 0;
  size_t bsmem = 0;
  CUtensorMap map_x1, map_g;  // weight gradient: input octets and gz
  WgradArgs wg;
};

}  // namespace

struct mg_unet {
  int L = 0, base = 0, nx = 0, ny = 0, nz = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error = "no error";
  char* arena = nullptr;
  int* err = nullptr;
  // tensors
  Tensor x0;                           // level-0 input, 16 channels
  Tensor d0[kMaxNetLevels];            // first down convolution
  Tensor d1[kMaxNetLevels];            // second down convolution (a channel range of cat[l] for l < L-1)
  Tensor pool[kMaxNetLevels];          // pooled input of level l >= 1
  Tensor cat[kMaxNetLevels];           // skip + upsampled, l < L-1
  Tensor u0[kMaxNetLevels], u1[kMaxNetLevels];
  float* xin = nullptr;                // FP32 input channels [3][V0] (staging)
  float* pred = nullptr;               // FP32 prediction [V0]
  float* head_w = nullptr;             // [c_0]
  float* head_b = nullptr;             // [1]
  float* nat = nullptr;                // FP32 staging for layer read-back
  size_t nat_elems = 0;
  std::vector<Conv> convs;             // parameter order: down0.0, down0.1, ..., down(L-1).1, up0.0, up0.1, ..., up(L-2).1
  long long n_params = 0;
  // training state: flat FP32 parameters, gradients and Adam moments
  float* theta = nullptr;
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long adam_t = 0;
  float* head_dw = nullptr;            // head gradients (in grad)
  Tensor gcat[kMaxNetLevels];          // gradient w.r.t. the concatenation, l < L-1
  Tensor gpool[kMaxNetLevels];         // gradient w.r.t. the pooled input, l >= 1
  float* gpred = nullptr;              // dL/dpred [V0]
  float* target = nullptr;             // training target [V0]
  float* wg_partial = nullptr;         // weight-gradient partial sums
  float* red_partial = nullptr;        // bias / head partial sums
  int red_blocks = 0;
  double* loss_part = nullptr;         // loss partial sums and the two totals
  double* loss_sums = nullptr;
  int loss_blocks = 0;
  double* feat_part = nullptr;         // feature partial sums
  double* feat_scale = nullptr;        // the patch's scale s
};

namespace {

thread_local std::string t_unet_error;

mg_status ufail(mg_unet* N, mg_status st, const std::string& msg) {
  if (N) N->last_error = msg;
  set_thread_error(msg.c_str());
  return st;
}

mg_status ucuda(mg_unet* N, cudaError_t e, const char* what) {
  return ufail(N, e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define UCK(N, call)                                      \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ucuda((N), e_, #call);  \
  } while (0)

#define UCKS(call)                \
  do {                            \
    mg_status s_ = (call);        \
    if (s_ != MG_OK) return s_;   \
  } while (0)

struct UGuard {
  int prev = -1;
  explicit UGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~UGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct Reserve {
  size_t used = 0;
  size_t take(size_t bytes) {
    const size_t o = (used + 255) & ~(size_t)255;
    used = o + bytes;
    return o;
  }
};

// Names the conv layers in parameter order.
std::string conv_name(const mg_unet* N, int i) {
  if (i < 2 * N->L) return "down" + std::to_string(i / 2) + "." + std::to_string(i % 2);
  const int j = i - 2 * N->L;
  return "up" + std::to_string(j / 2) + "." + std::to_string(j % 2);
}

mg_status setup_conv(mg_unet* N, Conv& C) {
  int bx, by, bz;
  conv_tile_box(C.in.W, C.in.H, C.in.D, &bx, &by, &bz);
  const int kc = conv_kc(C.cin_pad);
  ConvArgs& a = C.args;
  std::memset(&a, 0, sizeof(a));
  a.W = C.in.W;
  a.H = C.in.H;
  a.D = C.in.D;
  a.cin = C.cin_pad;
  a.cout = C.cout;
  a.kc = kc;
  a.bx = bx;
  a.by = by;
  a.bz = bz;
  a.ntx = (a.W + bx - 1) / bx;
  a.nty = (a.H + by - 1) / by;
  a.ntz = (a.D + bz - 1) / bz;
  a.w = C.wf;
  a.bias = C.b;
  a.relu = 1;
  a.out = C.out.p;
  a.out_stride = C.out.stride;
  a.out_off = C.out.off;
  a.err = N->err;
  conv_plan(a);
  C.smem = conv_smem_bytes(a);
  if (!(a.halo ? make_conv_input_map(&C.map_in, C.in.p, a.W, a.H, a.D, a.cin, 130, 3, 3, 2)
               : make_conv_input_map(&C.map_in, C.in.p, a.W, a.H, a.D, a.cin, bx, by, bz, kc)))
    return ufail(N, MG_ERR_CUDA, "tensor map of a convolution input was refused");
  return MG_OK;
}

// Backward of convolution C: the backward-data convolution (input C.gz,
// mirrored weights, output `to` masked by `mask` where the layer's input is
// a ReLU output) and the weight gradient's tensor maps and partition.
mg_status setup_conv_backward(mg_unet* N, Conv& C, const Tensor* to, const Tensor* mask) {
  int bx, by, bz;
  conv_tile_box(C.in.W, C.in.H, C.in.D, &bx, &by, &bz);
  const int T = ((C.in.W + bx - 1) / bx) * ((C.in.H + by - 1) / by) * ((C.in.D + bz - 1) / bz);
  // weight gradient
  if (!make_conv_input_map(&C.map_x1, C.in.p, C.in.W, C.in.H, C.in.D, C.cin_pad, bx, by, bz, 1) ||
      !make_conv_input_map(&C.map_g, C.gz.p, C.gz.W, C.gz.H, C.gz.D, C.cout, bx, by, bz, C.cout / 8))
    return ufail(N, MG_ERR_CUDA, "tensor map of a weight gradient was refused");
  WgradArgs& w = C.wg;
  std::memset(&w, 0, sizeof(w));
  w.W = C.in.W;
  w.H = C.in.H;
  w.D = C.in.D;
  w.cin = C.cin_pad;
  w.cout = C.cout;
  w.bx = bx;
  w.by = by;
  w.bz = bz;
  w.ntx = (w.W + bx - 1) / bx;
  w.nty = (w.H + by - 1) / by;
  w.ntz = (w.D + bz - 1) / bz;
  w.nmblk = (27 * C.cin_pad + 127) / 128;
  int ns = (2 * device_sms()) / w.nmblk;
  if (ns < 1) ns = 1;
  if (ns > T) ns = T;
  w.nsplit = ns;
  w.err = N->err;
  if (!to) return MG_OK;
  // backward data: K = cout (the gradient's channels), N = cin_pad
  const int kc = conv_kc(C.cout);
  ConvArgs& a = C.bargs;
  std::memset(&a, 0, sizeof(a));
  a.W = C.in.W;
  a.H = C.in.H;
  a.D = C.in.D;
  a.cin = C.cout;
  a.cout = C.cin_pad;
  a.kc = kc;
  a.bx = bx;
  a.by = by;
  a.bz = bz;
  a.ntx = w.ntx;
  a.nty = w.nty;
  a.ntz = w.ntz;
  a.w = C.wb;
  a.bias = nullptr;
  a.relu = 0;
  if (mask) {
    a.mask = mask->p;
    a.mask_stride = mask->stride;
    a.mask_off = mask->off;
  }
  a.out = to->p;
  a.out_stride = to->stride;
  a.out_off = to->off;
  a.err = N->err;
  conv_plan(a);
  C.bsmem = conv_smem_bytes(a);
  if (!(a.halo ? make_conv_input_map(&C.map_gz_bd, C.gz.p, a.W, a.H, a.D, a.cin, 130, 3, 3, 2)
               : make_conv_input_map(&C.map_gz_bd, C.gz.p, a.W, a.H, a.D, a.cin, bx, by, bz, kc)))
    return ufail(N, MG_ERR_CUDA, "tensor map of a backward convolution was refused");
  return MG_OK;
}

// The kernel's shared-memory limit is one attribute for all convolutions:
// set it to the largest need, then size each launch grid.
mg_status finish_convs(mg_unet* N) {
  size_t most = 0, most_w = 0;
  for (const Conv& C : N->convs) {
    most = C.smem > most ? C.smem : most;
    most = C.bsmem > most ? C.bsmem : most;
    const size_t ws = wgrad_smem_bytes(C.cout);
    most_w = ws > most_w ? ws : most_w;
  }
  UCK(N, init_conv_kernel(most));
  UCK(N, init_wgrad_kernel(most_w));
  for (Conv& C : N->convs) {
    C.grid = conv_grid(C.args, C.smem);
    if (C.wb) C.bgrid = conv_grid(C.bargs, C.bsmem);
  }
  return MG_OK;
}

mg_status check_err(mg_unet* N) {
  int e = 0;
  UCK(N, cudaStreamSynchronize(N->stream));
  UCK(N, cudaMemcpy(&e, N->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    UCK(N, cudaMemset(N->err, 0, sizeof(int)));
    return ufail(N, MG_ERR_INTERNAL, "network kernel: a wait on an asynchronous copy or MMA did not complete in time");
  }
  return MG_OK;
}

mg_status forward(mg_unet* N) {
  cudaStream_t s = N->stream;
  const int L = N->L;
  for (int l = 0; l < L; ++l) {
    if (l > 0) {
      const Tensor& src = N->d1[l - 1];
      const Tensor& dst = N->pool[l];
      UCK(N, launch_avg_pool(src.p, src.stride, src.off, dst.W, dst.H, dst.D, dst.c, dst.p, dst.stride, dst.off, s));
    }
    for (int j = 0; j < 2; ++j) {
      Conv& C = N->convs[2 * l + j];
      UCK(N, launch_conv(C.map_in, C.args, C.grid, s));
    }
  }
  for (int l = L - 2; l >= 0; --l) {
    const Tensor& prev = l == L - 2 ? N->d1[L - 1] : N->u1[l + 1];
    const Tensor& cat = N->cat[l];
    UCK(N, launch_upsample(prev.p, prev.stride, prev.off, prev.W, prev.H, prev.D, prev.c, cat.p, cat.stride,
                           N->d1[l].c, s));
    for (int j = 0; j < 2; ++j) {
      Conv& C = N->convs[2 * L + 2 * l + j];
      UCK(N, launch_conv(C.map_in, C.args, C.grid, s));
    }
  }
  const Tensor& top = L >= 2 ? N->u1[0] : N->d1[0];
  UCK(N, launch_head(top.p, top.c, N->head_w, N->head_b, N->x0.p, N->x0.voxels(), N->pred, s));
  return MG_OK;
}

mg_status conv_weight_grad(mg_unet* N, Conv& C) {
  cudaStream_t s = N->stream;
  WgradArgs a = C.wg;
  a.partial = N->wg_partial;
  UCK(N, launch_wgrad(C.map_x1, C.map_g, a, s));
  UCK(N, launch_wgrad_reduce(N->wg_partial, a.nsplit, a.nmblk * 128, C.cin_pad, C.cin, C.cout, C.dw, s));
  UCK(N, launch_bias_grad(C.gz.p, C.cout, C.gz.voxels(), N->red_partial, N->red_blocks, C.db, s));
  return MG_OK;
}

// Backward pass from N->gpred (dL/dpred): every parameter's gradient into
// N->grad, through the layers in reverse order of the forward pass.
mg_status backward(mg_unet* N) {
  cudaStream_t s = N->stream;
  const int L = N->L;
  auto cidx_down = [&](int l, int j) { return 2 * l + j; };
  auto cidx_up = [&](int l, int j) { return 2 * L + 2 * l + j; };
  Conv& topc = N->convs[L >= 2 ? cidx_up(0, 1) : cidx_down(0, 1)];
  UCK(N, launch_head_backward(N->gpred, N->x0.p, topc.out.p, N->base, N->head_w, N->x0.voxels(), topc.gz.p,
                              N->red_partial, N->red_blocks, N->head_dw, s));
  for (int l = 0; l < L - 1; ++l) {
    for (int j = 1; j >= 0; --j) {
      Conv& C = N->convs[cidx_up(l, j)];
      UCKS(conv_weight_grad(N, C));
      UCK(N, launch_conv(C.map_gz_bd, C.bargs, C.bgrid, s));
    }
    // the upsampled part of the concatenation's gradient is the gradient of
    // the level below's output (already masked by its ReLU)
    Conv& below = N->convs[l == L - 2 ? cidx_down(L - 1, 1) : cidx_up(l + 1, 1)];
    const Tensor& gc = N->gcat[l];
    UCK(N, launch_upsample_backward(gc.p, gc.stride, N->d1[l].c, below.gz.W, below.gz.H, below.gz.D, below.gz.c,
                                    below.gz.p, s));
  }
  for (int l = L - 1; l >= 0; --l) {
    Conv& C1 = N->convs[cidx_down(l, 1)];
    if (l < L - 1) {
      const Tensor& gc = N->gcat[l];
      const Tensor& gp = N->gpool[l + 1];
      UCK(N, launch_skip_pool_combine(gc.p, gc.stride, N->d1[l].p, N->d1[l].stride, gp.p, C1.gz.W, C1.gz.H, C1.gz.D,
                                      C1.gz.c, C1.gz.p, s));
    }
    UCKS(conv_weight_grad(N, C1));
    UCK(N, launch_conv(C1.map_gz_bd, C1.bargs, C1.bgrid, s));
    Conv& C0 = N->convs[cidx_down(l, 0)];
    UCKS(conv_weight_grad(N, C0));
    if (l > 0) UCK(N, launch_conv(C0.map_gz_bd, C0.bargs, C0.bgrid, s));
  }
  return MG_OK;
}

// Re-rounds the BF16 working weights from the FP32 masters.
mg_status pack_all(mg_unet* N) {
  for (Conv& C : N->convs) {
    UCK(N, launch_pack_weights(C.w, C.cout, C.cin, C.cin_pad, false, C.wf, N->stream));
    if (C.wb) UCK(N, launch_pack_weights(C.w, C.cout, C.cin, C.cin_pad, true, C.wb, N->stream));
  }
  return MG_OK;
}

void destroy_unet(mg_unet* N) {
  if (!N) return;
  UGuard g(N->device);
  if (N->stream) cudaStreamSynchronize(N->stream);
  if (N->arena) cudaFree(N->arena);
  if (N->own_stream && N->stream) cudaStreamDestroy(N->stream);
  delete N;
}

// copy `bytes` between a caller buffer and device memory
mg_status copy_io(mg_unet* N, void* dst, const void* src, size_t bytes, bool to_device, mg_mem where) {
  if (where == MG_MEM_DEVICE) {
    const void* user = to_device ? src : dst;
    if (!is_device_ptr(user, N->device))
      return ufail(N, MG_ERR_INVALID_ARG, "an MG_MEM_DEVICE buffer is not device memory of the network's GPU");
    UCK(N, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, N->stream));
    return MG_OK;
  }
  UCK(N, cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, N->stream));
  UCK(N, cudaStreamSynchronize(N->stream));
  return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_unet_create(int levels, int base, int nx, int ny, int nz, void* cuda_stream, mg_unet** out) {
  if (out) *out = nullptr;
  if (!out) return ufail(nullptr, MG_ERR_INVALID_ARG, "null output");
  if (levels < 1 || levels > kMaxNetLevels || base < 16 || base % 16 || base << (levels - 1) > 128)
    return ufail(nullptr, MG_ERR_INVALID_ARG, "levels must be 1..6 and base a multiple of 16 with base 2^(levels-1) <= 128");
  const int div = 1 << (levels - 1);
  if (nx < 1 || ny < 1 || nz < 1 || nx % div || ny % div || nz % div || nx > 1024 || ny > 1024 || nz > 1024)
    return ufail(nullptr, MG_ERR_INVALID_ARG, "dimensions must be 1..1024 and divisible by 2^(levels-1)");
  mg_unet* N = new mg_unet();
  N->L = levels;
  N->base = base;
  N->nx = nx;
  N->ny = ny;
  N->nz = nz;
  if (cudaGetDevice(&N->device) != cudaSuccess) {
    delete N;
    return ufail(nullptr, MG_ERR_CUDA, "no CUDA device");
  }
  if (cuda_stream) {
    N->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreate(&N->stream) != cudaSuccess) {
      delete N;
      return ufail(nullptr, MG_ERR_CUDA, "cudaStreamCreate");
    }
    N->own_stream = true;
  }
  const int L = levels;
  std::vector<int> ch(L);
  for (int l = 0; l < L; ++l) ch[l] = base << l;
  // tensors and their arena offsets
  Reserve R;
  struct Pending {
    Tensor* t;
    size_t off;
  };
  std::vector<Pending> pend;
  auto tensor = [&](Tensor& t, int level, int stride, int off, int c, bool alloc) {
    t.W = nx >> level;
    t.H = ny >> level;
    t.D = nz >> level;
    t.stride = stride;
    t.off = off;
    t.c = c;
    if (alloc) pend.push_back({&t, R.take(sizeof(__nv_bfloat16) * (size_t)t.voxels() * stride)});
  };
  tensor(N->x0, 0, 16, 0, 16, true);
  for (int l = 0; l < L; ++l) {
    if (l > 0) tensor(N->pool[l], l, ch[l - 1], 0, ch[l - 1], true);
    tensor(N->d0[l], l, ch[l], 0, ch[l], true);
    if (l < L - 1) {
      tensor(N->cat[l], l, ch[l] + ch[l + 1], 0, ch[l] + ch[l + 1], true);
      tensor(N->d1[l], l, ch[l] + ch[l + 1], 0, ch[l], false);  // shares cat[l]'s buffer
    } else {
      tensor(N->d1[l], l, ch[l], 0, ch[l], true);
    }
  }
  for (int l = 0; l < L - 1; ++l) {
    tensor(N->u0[l], l, ch[l], 0, ch[l], true);
    tensor(N->u1[l], l, ch[l], 0, ch[l], true);
  }
  const long long V0 = (long long)nx * ny * nz;
  const size_t o_xin = R.take(sizeof(float) * 3 * V0);
  const size_t o_pred = R.take(sizeof(float) * V0);
  N->nat_elems = (size_t)V0 * (size_t)(ch[0] + (L > 1 ? ch[1] : 0) + 16);
  const size_t o_nat = R.take(sizeof(float) * N->nat_elems);
  const size_t o_err = R.take(sizeof(int) * 4);
  // convolutions
  struct ConvPlan {
    int cin, cout, level;
  };
  std::vector<ConvPlan> plan;
  for (int l = 0; l < L; ++l) {
    plan.push_back({l == 0 ? 3 : ch[l - 1], ch[l], l});
    plan.push_back({ch[l], ch[l], l});
  }
  for (int l = 0; l < L - 1; ++l) {
    plan.push_back({ch[l] + ch[l + 1], ch[l], l});
    plan.push_back({ch[l], ch[l], l});
  }
  N->convs.resize(plan.size());
  std::vector<size_t> o_wf(plan.size()), o_wb(plan.size()), o_gz(plan.size());
  N->n_params = 0;
  size_t wg_floats = 0;
  for (size_t i = 0; i < plan.size(); ++i) {
    Conv& C = N->convs[i];
    C.cin = plan[i].cin;
    C.cin_pad = (C.cin + 15) / 16 * 16;
    C.cout = plan[i].cout;
    C.level = plan[i].level;
    C.off_w = N->n_params;
    C.off_b = C.off_w + (long long)C.cout * C.cin * 27;
    N->n_params = C.off_b + C.cout;
    o_wf[i] = R.take(sizeof(__nv_bfloat16) * 27 * (size_t)C.cout * C.cin_pad);
    o_wb[i] = i > 0 ? R.take(sizeof(__nv_bfloat16) * 27 * (size_t)C.cout * C.cin_pad) : 0;
    const int l = C.level;
    const long long Vl = (long long)(nx >> l) * (ny >> l) * (nz >> l);
    o_gz[i] = R.take(sizeof(__nv_bfloat16) * (size_t)Vl * C.cout);
    // weight-gradient partial sums (the partition of setup_conv_backward)
    int bx, by, bz;
    conv_tile_box(nx >> l, ny >> l, nz >> l, &bx, &by, &bz);
    const int T = (((nx >> l) + bx - 1) / bx) * (((ny >> l) + by - 1) / by) * (((nz >> l) + bz - 1) / bz);
    const int nmblk = (27 * C.cin_pad + 127) / 128;
    int ns = (2 * device_sms()) / nmblk;
    if (ns < 1) ns = 1;
    if (ns > T) ns = T;
    const size_t wf = (size_t)ns * nmblk * 128 * C.cout;
    wg_floats = wf > wg_floats ? wf : wg_floats;
  }
  const long long off_head = N->n_params;
  N->n_params += ch[0] + 1;
  const size_t o_theta = R.take(sizeof(float) * (size_t)N->n_params);
  const size_t o_grad = R.take(sizeof(float) * (size_t)N->n_params);
  const size_t o_m = R.take(sizeof(float) * (size_t)N->n_params);
  const size_t o_v = R.take(sizeof(float) * (size_t)N->n_params);
  for (int l = 0; l + 1 < L; ++l) tensor(N->gcat[l], l, ch[l] + ch[l + 1], 0, ch[l] + ch[l + 1], true);
  for (int l = 1; l < L; ++l) tensor(N->gpool[l], l, ch[l - 1], 0, ch[l - 1], true);
  const size_t o_gpred = R.take(sizeof(float) * V0);
  const size_t o_target = R.take(sizeof(float) * V0);
  const size_t o_wgp = R.take(sizeof(float) * wg_floats);
  N->red_blocks = 256;
  const size_t o_red = R.take(sizeof(float) * (size_t)N->red_blocks * (128 + 1));
  N->loss_blocks = 512;
  const size_t o_lp = R.take(sizeof(double) * (2 * (size_t)N->loss_blocks + 2));
  const size_t o_fp = R.take(sizeof(double) * (4 * (size_t)N->loss_blocks + 2));

  cudaError_t e = dev_malloc((void**)&N->arena, R.used);
  if (e != cudaSuccess) {
    N->arena = nullptr;
    mg_status st = ucuda(nullptr, e, "cudaMalloc(network arena)");
    destroy_unet(N);
    return st;
  }
  char* base_p = N->arena;
  for (auto& p : pend) p.t->p = (__nv_bfloat16*)(base_p + p.off);
  for (int l = 0; l < L - 1; ++l) N->d1[l].p = N->cat[l].p;
  N->xin = (float*)(base_p + o_xin);
  N->pred = (float*)(base_p + o_pred);
  N->nat = (float*)(base_p + o_nat);
  N->err = (int*)(base_p + o_err);
  N->theta = (float*)(base_p + o_theta);
  N->grad = (float*)(base_p + o_grad);
  N->adam_m = (float*)(base_p + o_m);
  N->adam_v = (float*)(base_p + o_v);
  N->head_w = N->theta + off_head;
  N->head_b = N->theta + off_head + ch[0];
  N->head_dw = N->grad + off_head;
  N->gpred = (float*)(base_p + o_gpred);
  N->target = (float*)(base_p + o_target);
  N->wg_partial = (float*)(base_p + o_wgp);
  N->red_partial = (float*)(base_p + o_red);
  N->loss_part = (double*)(base_p + o_lp);
  N->loss_sums = N->loss_part + 2 * N->loss_blocks;
  N->feat_part = (double*)(base_p + o_fp);
  N->feat_scale = N->feat_part + 4 * N->loss_blocks;
  mg_status st = MG_OK;
  if (cudaMemsetAsync(N->arena, 0, R.used, N->stream) != cudaSuccess) st = ufail(N, MG_ERR_CUDA, "arena reset");
  for (size_t i = 0; i < plan.size(); ++i) {
    Conv& C = N->convs[i];
    C.gz.p = (__nv_bfloat16*)(base_p + o_gz[i]);
    C.gz.W = nx >> C.level;
    C.gz.H = ny >> C.level;
    C.gz.D = nz >> C.level;
    C.gz.stride = C.gz.c = C.cout;
    C.gz.off = 0;
  }
  for (size_t i = 0; i < plan.size() && st == MG_OK; ++i) {
    Conv& C = N->convs[i];
    C.w = N->theta + C.off_w;
    C.b = N->theta + C.off_b;
    C.dw = N->grad + C.off_w;
    C.db = N->grad + C.off_b;
    C.wf = (__nv_bfloat16*)(base_p + o_wf[i]);
    C.wb = i > 0 ? (__nv_bfloat16*)(base_p + o_wb[i]) : nullptr;
    const int l = C.level;
    const bool down = (int)i < 2 * L;
    const int j = (int)i % 2;
    if (down) {
      C.in = j == 0 ? (l == 0 ? N->x0 : N->pool[l]) : N->d0[l];
      C.out = j == 0 ? N->d0[l] : N->d1[l];
    } else {
      C.in = j == 0 ? N->cat[l] : N->u0[l];
      C.out = j == 0 ? N->u0[l] : N->u1[l];
    }
    st = setup_conv(N, C);
  }
  for (size_t i = 0; i < plan.size() && st == MG_OK; ++i) {
    Conv& C = N->convs[i];
    const int l = C.level;
    const int j = (int)i % 2;
    if ((int)i < 2 * L) {
      if (j == 0) st = setup_conv_backward(N, C, l == 0 ? nullptr : &N->gpool[l], nullptr);
      else st = setup_conv_backward(N, C, &N->convs[i - 1].gz, &N->d0[l]);
    } else {
      if (j == 0) st = setup_conv_backward(N, C, &N->gcat[l], &N->cat[l]);
      else st = setup_conv_backward(N, C, &N->convs[i - 1].gz, &N->u0[l]);
    }
  }
  if (st == MG_OK) st = finish_convs(N);
  if (st == MG_OK && cudaStreamSynchronize(N->stream) != cudaSuccess) st = ufail(N, MG_ERR_CUDA, "network setup");
  if (st != MG_OK) {
    std::string msg = N->last_error;
    destroy_unet(N);
    set_thread_error(msg.c_str());
    return st;
  }
  *out = N;
  return MG_OK;
}

mg_status mg_unet_destroy(mg_unet* N) {
  destroy_unet(N);
  return MG_OK;
}

mg_status mg_unet_num_params(const mg_unet* N, long long* n) {
  if (!N || !n) return ufail(nullptr, MG_ERR_INVALID_ARG, "null argument");
  *n = N->n_params;
  return MG_OK;
}

mg_status mg_unet_set_params(mg_unet* N, const double* p, mg_mem where) {
  if (!N || !p) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  UGuard g(N->device);
  std::vector<double> h((size_t)N->n_params);
  if (where == MG_MEM_DEVICE) {
    if (!is_device_ptr(p, N->device))
      return ufail(N, MG_ERR_INVALID_ARG, "an MG_MEM_DEVICE buffer is not device memory of the network's GPU");
    UCK(N, cudaMemcpy(h.data(), p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(h.data(), p, sizeof(double) * h.size());
  }
  std::vector<float> f(h.begin(), h.end());
  UCK(N, cudaMemcpy(N->theta, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice));
  UCKS(pack_all(N));
  UCK(N, cudaStreamSynchronize(N->stream));
  return MG_OK;
}

mg_status mg_unet_get_params(mg_unet* N, double* p, mg_mem where) {
  if (!N || !p) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  UGuard g(N->device);
  UCK(N, cudaStreamSynchronize(N->stream));
  std::vector<float> f((size_t)N->n_params);
  UCK(N, cudaMemcpy(f.data(), N->theta, sizeof(float) * f.size(), cudaMemcpyDeviceToHost));
  std::vector<double> h(f.begin(), f.end());
  if (where == MG_MEM_DEVICE) {
    if (!is_device_ptr(p, N->device))
      return ufail(N, MG_ERR_INVALID_ARG, "an MG_MEM_DEVICE buffer is not device memory of the network's GPU");
    UCK(N, cudaMemcpy(p, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
  } else {
    std::memcpy(p, h.data(), sizeof(double) * h.size());
  }
  return MG_OK;
}

mg_status mg_unet_forward(mg_unet* N, const float* x, mg_mem where, float* pred, mg_mem pred_where) {
  if (!N || !x) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  UGuard g(N->device);
  const long long V0 = N->x0.voxels();
  UCKS(copy_io(N, N->xin, x, sizeof(float) * 3 * V0, true, where));
  UCK(N, launch_input_to_bf16(N->xin, V0, N->x0.p, N->stream));
  UCKS(forward(N));
  UCKS(check_err(N));
  if (pred) UCKS(copy_io(N, pred, N->pred, sizeof(float) * V0, false, pred_where));
  return MG_OK;
}

mg_status mg_unet_backward(mg_unet* N, const float* g_pred, mg_mem where) {
  if (!N || !g_pred) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  UGuard g(N->device);
  UCKS(copy_io(N, N->gpred, g_pred, sizeof(float) * N->x0.voxels(), true, where));
  UCKS(backward(N));
  return check_err(N);
}

mg_status mg_unet_get_grads(mg_unet* N, double* out, mg_mem where) {
  if (!N || !out) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  UGuard g(N->device);
  UCK(N, cudaStreamSynchronize(N->stream));
  std::vector<float> f((size_t)N->n_params);
  UCK(N, cudaMemcpy(f.data(), N->grad, sizeof(float) * f.size(), cudaMemcpyDeviceToHost));
  std::vector<double> h(f.begin(), f.end());
  if (where == MG_MEM_DEVICE) {
    if (!is_device_ptr(out, N->device))
      return ufail(N, MG_ERR_INVALID_ARG, "an MG_MEM_DEVICE buffer is not device memory of the network's GPU");
    UCK(N, cudaMemcpy(out, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
  } else {
    std::memcpy(out, h.data(), sizeof(double) * h.size());
  }
  return MG_OK;
}

mg_status mg_unet_adam_step(mg_unet* N, double lr, double beta1, double beta2, double eps) {
  if (!N || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return ufail(N, MG_ERR_INVALID_ARG, "bad Adam parameters");
  UGuard g(N->device);
  N->adam_t += 1;
  const double bc1 = 1.0 - std::pow(beta1, (double)N->adam_t), bc2 = 1.0 - std::pow(beta2, (double)N->adam_t);
  UCK(N, launch_adam(N->theta, N->grad, N->adam_m, N->adam_v, N->n_params, (float)lr, (float)beta1, (float)beta2,
                     (float)eps, (float)bc1, (float)bc2, N->stream));
  UCKS(pack_all(N));
  return MG_OK;
}

mg_status mg_unet_train_step(mg_unet* N, const float* x, const float* y, mg_mem where, double lr, double* loss) {
  if (!N || !x || !y) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  UGuard g(N->device);
  const long long V0 = N->x0.voxels();
  UCKS(copy_io(N, N->xin, x, sizeof(float) * 3 * V0, true, where));
  UCKS(copy_io(N, N->target, y, sizeof(float) * V0, true, where));
  UCK(N, launch_input_to_bf16(N->xin, V0, N->x0.p, N->stream));
  UCKS(forward(N));
  UCK(N, launch_loss(N->pred, N->target, N->x0.p, V0, N->loss_part, N->loss_blocks, N->loss_sums, N->gpred, N->stream));
  UCKS(backward(N));
  UCKS(mg_unet_adam_step(N, lr, 0.9, 0.999, 1e-8));
  if (loss) {
    double sums[2];
    UCK(N, cudaMemcpyAsync(sums, N->loss_sums, sizeof(sums), cudaMemcpyDeviceToHost, N->stream));
    UCKS(check_err(N));
    *loss = sums[0] > 0 ? sums[1] / sums[0] : 0.0;
    return MG_OK;
  }
  return MG_OK;
}

static mg_status patch_inputs(mg_unet* N, const int8_t* mask, const double* rho, const double* bx, const double* by,
                              const double* bz, double h) {
  if (!mask || !rho || !(h > 0)) return ufail(N, MG_ERR_INVALID_ARG, "null mask or rho, or h <= 0");
  for (const void* p : {(const void*)mask, (const void*)rho, (const void*)bx, (const void*)by, (const void*)bz})
    if (p && !is_device_ptr(p, N->device))
      return ufail(N, MG_ERR_INVALID_ARG, "patch buffers must be device memory of the network's GPU");
  UCK(N, launch_features(mask, rho, bx, by, bz, N->nx, N->ny, N->nz, h, N->feat_part, N->loss_blocks, N->feat_scale,
                         N->xin, N->stream));
  UCK(N, launch_input_to_bf16(N->xin, N->x0.voxels(), N->x0.p, N->stream));
  return MG_OK;
}

mg_status mg_unet_features(mg_unet* N, const int8_t* mask, const double* rho, const double* bx, const double* by,
                           const double* bz, double h, float* x, mg_mem where, double* scale) {
  if (!N) return ufail(N, MG_ERR_INVALID_ARG, "null network");
  UGuard g(N->device);
  UCKS(patch_inputs(N, mask, rho, bx, by, bz, h));
  if (x) UCKS(copy_io(N, x, N->xin, sizeof(float) * 3 * N->x0.voxels(), false, where));
  if (scale) UCK(N, cudaMemcpy(scale, N->feat_scale, sizeof(double), cudaMemcpyDeviceToHost));
  return MG_OK;
}

mg_status mg_unet_predict(mg_unet* N, const int8_t* mask, const double* rho, const double* bx, const double* by,
                          const double* bz, double h, double* phi) {
  if (!N || !phi) return ufail(N, MG_ERR_INVALID_ARG, "null network or output");
  UGuard g(N->device);
  if (!is_device_ptr(phi, N->device)) return ufail(N, MG_ERR_INVALID_ARG, "phi must be device memory");
  UCKS(patch_inputs(N, mask, rho, bx, by, bz, h));
  UCKS(forward(N));
  UCK(N, launch_scale_prediction(N->pred, N->x0.voxels(), N->feat_scale, phi, N->stream));
  return MG_OK;
}

mg_status mg_unet_train_patch(mg_unet* N, const int8_t* mask, const double* rho, const double* bx, const double* by,
                              const double* bz, double h, const double* phi, double lr, double* loss) {
  if (!N || !phi) return ufail(N, MG_ERR_INVALID_ARG, "null network or target");
  UGuard g(N->device);
  if (!is_device_ptr(phi, N->device)) return ufail(N, MG_ERR_INVALID_ARG, "phi must be device memory");
  const long long V0 = N->x0.voxels();
  UCKS(patch_inputs(N, mask, rho, bx, by, bz, h));
  UCK(N, launch_scale_target(phi, V0, N->feat_scale, N->target, N->stream));
  UCKS(forward(N));
  UCK(N, launch_loss(N->pred, N->target, N->x0.p, V0, N->loss_part, N->loss_blocks, N->loss_sums, N->gpred, N->stream));
  UCKS(backward(N));
  UCKS(mg_unet_adam_step(N, lr, 0.9, 0.999, 1e-8));
  if (loss) {
    double sums[2];
    UCK(N, cudaMemcpyAsync(sums, N->loss_sums, sizeof(sums), cudaMemcpyDeviceToHost, N->stream));
    UCKS(check_err(N));
    *loss = sums[0] > 0 ? sums[1] / sums[0] : 0.0;
  }
  return MG_OK;
}

mg_status mg_unet_layer_output(mg_unet* N, int layer, float* out, mg_mem where) {
  if (!N || !out) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  if (layer < 0 || layer >= (int)N->convs.size()) return ufail(N, MG_ERR_INVALID_ARG, "layer out of range");
  UGuard g(N->device);
  const Tensor& t = N->convs[layer].out;
  const size_t n = (size_t)t.c * t.voxels();
  if (n > N->nat_elems) return ufail(N, MG_ERR_INTERNAL, "read-back staging too small");
  UCK(N, launch_tensor_to_natural(t.p, t.stride, t.off, t.c, t.voxels(), N->nat, N->stream));
  return copy_io(N, out, N->nat, sizeof(float) * n, false, where);
}

mg_status mg_unet_layer_grad(mg_unet* N, int layer, float* out, mg_mem where) {
  if (!N || !out) return ufail(N, MG_ERR_INVALID_ARG, "null argument");
  if (layer < 0 || layer >= (int)N->convs.size()) return ufail(N, MG_ERR_INVALID_ARG, "layer out of range");
  UGuard g(N->device);
  const Tensor& t = N->convs[layer].gz;
  const size_t n = (size_t)t.c * t.voxels();
  if (n > N->nat_elems) return ufail(N, MG_ERR_INTERNAL, "read-back staging too small");
  UCK(N, launch_tensor_to_natural(t.p, t.stride, t.off, t.c, t.voxels(), N->nat, N->stream));
  return copy_io(N, out, N->nat, sizeof(float) * n, false, where);
}

mg_status mg_unet_layer_info(const mg_unet* N, int layer, int* dims4) {
  if (!N || !dims4) return ufail(nullptr, MG_ERR_INVALID_ARG, "null argument");
  if (layer < 0 || layer >= (int)N->convs.size()) return ufail(nullptr, MG_ERR_INVALID_ARG, "layer out of range");
  const Tensor& t = N->convs[layer].out;
  dims4[0] = t.c;
  dims4[1] = t.D;
  dims4[2] = t.H;
  dims4[3] = t.W;
  return MG_OK;
}

const char* mg_unet_last_error(const mg_unet* N) { return N ? N->last_error.c_str() : mg_last_error(nullptr); }

}  // extern "C"
