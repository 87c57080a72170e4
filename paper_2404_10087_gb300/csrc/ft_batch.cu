// Batched persistent epoch (include/ft.h, "batches"): many independent
// tensors, grouped by kernel class, one persistent factor kernel and one
// persistent core kernel per class over fixed-size work units, one finalize
// over every tensor, the whole epoch captured once as a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "ft.h"
#include "ft_device.cuh"
#include "ft_internal.h"

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Candidate launch shapes of the autotuner (warp tiles per unit; the smallest
// sizes the workspace).
constexpr int kUnitTiles[] = {64, 256, 1024};
constexpr int kDefaultUnitTiles = 256;
constexpr int kMinUnitTiles = 64;

struct BatchFinalDesc {
  float *B[FT_MAXN];
  int J[FT_MAXN];
  int N, K, R;
  int nunits;           // units of the tensor (consecutive partials)
  int64_t poff;         // float offset of the first unit's partial
  int64_t elem_begin;   // first element of this tensor in the finalize index space
  float inv_nnz;
};

struct FinalArgs {
  const BatchFinalDesc *d;
  int ntensors;
  int64_t total;
  const float *partial;
  const float *hyper;
};

// Per-tensor core finalize: G = sum over the tensor's unit partials
// (compensated, in a fixed order), B <- B - lr_b (G / nnz + lambda_b B)
// (Algorithm 5, last step).  One warp per element: lane l sums the partials
// of units l, l + 32, ... in order, then a fixed xor tree combines the lanes
// and lane 0 holds the result - the same order on every run.
__global__ void k_batch_finalize(const FinalArgs a) {
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.total) return;
  int lo = 0, hi = a.ntensors - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (a.d[mid].elem_begin <= warp) lo = mid;
    else hi = mid - 1;
  }
  const BatchFinalDesc &d = a.d[lo];
  const int64_t local = warp - d.elem_begin;
  const int KK = d.K * d.K;
  const int n = int(local / KK), j = int((local % KK) / d.K), r = int(local % d.K);
  if (j >= d.J[n] || r >= d.R) return;
  const int64_t stride = 2LL * d.N * KK;
  float s = 0.f, c = 0.f;
  for (int q = lane; q < d.nunits; q += 32) {
    const float2 pp = *reinterpret_cast<const float2 *>(a.partial + d.poff + q * stride + 2 * local);
    ft::neumaier_add(s, c, pp.x);
    c += pp.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
    ft::neumaier_add(s, c, s2);
    c += c2;
  }
  if (lane != 0) return;
  const float G = s + c;
  float *b = d.B[n] + j * d.R + r;
  const float bv = *b;
  *b = bv - a.hyper[2] * fmaf(G, d.inv_nnz, a.hyper[3] * bv);
}

__global__ void k_set_hyper(float *h, float lr_a, float lam_a, float lr_b, float lam_b) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    h[0] = lr_a;
    h[1] = lam_a;
    h[2] = lr_b;
    h[3] = lam_b;
  }
}

struct ValidateOne {
  const int32_t *idx[FT_MAXN];
  int64_t I[FT_MAXN];
  int N;
  const float *vals;
  int64_t nnz;
  int *err;
};

__global__ void k_batch_validate(const ValidateOne v) {
  int bad = 0;
  for (int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; m < v.nnz;
       m += int64_t(gridDim.x) * blockDim.x) {
    for (int n = 0; n < v.N; ++n) {
      const int32_t i = v.idx[n][m];
      if (i < 0 || i >= v.I[n]) bad |= ft::ERRBIT_INDEX;
    }
    if (!isfinite(v.vals[m])) bad |= ft::ERRBIT_VALUE;
  }
  bad = __reduce_or_sync(ft::FULL, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(v.err, bad);
}

struct ErrFinal {
  const double *part;
  int nparts;
  int64_t n;
  double *out3;
};

__global__ void k_batch_errors_final(const ErrFinal a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double se = 0.0, ae = 0.0;
  for (int q = 0; q < a.nparts; ++q) { se += a.part[2 * q]; ae += a.part[2 * q + 1]; }
  a.out3[0] = a.n > 0 ? sqrt(se / double(a.n)) : 0.0;
  a.out3[1] = a.n > 0 ? ae / double(a.n) : 0.0;
  a.out3[2] = se;
}

bool kernel_set(int N, int K, int prec, ft::KernelSet *ks) { return ft_kernel_set(N, K, prec, ks); }

int occupancy(const void *fn, int threads, size_t smem) {
  int nb = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) return 0;
  return nb;
}

struct TensorInfo {
  int N, R, K;
  int J[FT_MAXN];
  int64_t I[FT_MAXN];
  int64_t nnz, ntiles;
  const int32_t *idx[FT_MAXN];
  const float *vals;
  float *A[FT_MAXN];
  float *B[FT_MAXN];
};

struct ClassInfo {
  int N, K;
  std::vector<int> tensors;
  ft::KernelSet ks;
  int occ_factor = 1, occ_core = 1;
  int unit_tiles = kDefaultUnitTiles;
  int ctas_per_sm = 0;       // 0: occupancy limit
  int64_t unit_first = 0, nunits = 0;
};

struct Layout {
  size_t off_hyper = 0, off_err = 0, off_tensors = 0, off_units = 0, off_final = 0;
  size_t off_partial = 0, off_errpart = 0, total = 0;
  int64_t max_units = 0, max_partial_floats = 0;
  int grid_eval = 0;
};

ft_status plan_batch(int nt, const ft_tensor_desc *d, const ft_config *cfg_in, ft_config *cfg,
                     std::vector<TensorInfo> *tensors, std::vector<ClassInfo> *classes, Layout *L,
                     int *num_sms) {
  if (nt < 1 || !d) return FT_ERR_ARG;
  ft_config_default(cfg);
  if (cfg_in) *cfg = *cfg_in;
  if (cfg->precision < FT_FP32 || cfg->precision > FT_BF16) return FT_ERR_ARG;
  if (cfg->scatter != FT_HOGWILD) return FT_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FT_ERR_CUDA;
  if (cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FT_ERR_CUDA;
  tensors->assign(size_t(nt), TensorInfo{});
  std::map<std::pair<int, int>, int> cls_of;
  classes->clear();
  for (int t = 0; t < nt; ++t) {
    const ft_tensor_desc &x = d[t];
    TensorInfo &ti = (*tensors)[size_t(t)];
    if (x.N < 1 || x.N > FT_MAX_ORDER || x.R < 1 || x.R > FT_MAX_RANK || !x.I || !x.J) return FT_ERR_SHAPE;
    if (x.nnz < 0 || x.nnz > INT32_MAX) return FT_ERR_ARG;
    if ((x.nnz > 0 && (!x.idx || !x.vals)) || !x.A || !x.B) return FT_ERR_ARG;
    int maxr = x.R;
    for (int n = 0; n < x.N; ++n) {
      if (x.J[n] < 1 || x.J[n] > FT_MAX_RANK || x.I[n] < 1 || x.I[n] > INT32_MAX) return FT_ERR_SHAPE;
      if ((x.nnz > 0 && !x.idx[n]) || !x.A[n] || !x.B[n]) return FT_ERR_ARG;
      maxr = std::max(maxr, x.J[n]);
      ti.J[n] = x.J[n];
      ti.I[n] = x.I[n];
      ti.idx[n] = x.nnz > 0 ? x.idx[n] : nullptr;
      ti.A[n] = x.A[n];
      ti.B[n] = x.B[n];
    }
    ti.N = x.N;
    ti.R = x.R;
    ti.K = maxr <= 16 ? 16 : 32;
    if (ti.N * ti.K > 160) return FT_ERR_SHAPE;
    ti.nnz = x.nnz;
    ti.ntiles = (x.nnz + FT_TILE - 1) / FT_TILE;
    ti.vals = x.vals;
    auto key = std::make_pair(ti.N, ti.K);
    auto it = cls_of.find(key);
    if (it == cls_of.end()) {
      ClassInfo c;
      c.N = ti.N;
      c.K = ti.K;
      if (!kernel_set(ti.N, ti.K, cfg->precision, &c.ks)) return FT_ERR_SHAPE;
      c.occ_factor = occupancy(c.ks.batch_factor, c.ks.batch_factor_threads, c.ks.factor_smem);
      c.occ_core = occupancy(c.ks.batch_core, c.ks.batch_core_threads, c.ks.batch_core_smem);
      if (c.occ_factor < 1 || c.occ_core < 1) return FT_ERR_CUDA;
      it = cls_of.emplace(key, int(classes->size())).first;
      classes->push_back(c);
    }
    (*classes)[size_t(it->second)].tensors.push_back(t);
  }
  // workspace, sized for the smallest unit
  int64_t max_units = 0, max_partial = 0;
  for (const TensorInfo &ti : *tensors) {
    const int64_t u = std::max<int64_t>(1, (ti.ntiles + kMinUnitTiles - 1) / kMinUnitTiles);
    max_units += u;
    max_partial += u * 2LL * ti.N * ti.K * ti.K;
  }
  int occ_eval = 8;
  L->grid_eval = *num_sms * occ_eval;
  size_t off = 0;
  L->off_hyper = off;   off += align_up(4 * sizeof(float));
  L->off_err = off;     off += align_up(sizeof(int) * 16 + sizeof(double) * 4);
  L->off_tensors = off; off += align_up(sizeof(ft::EpochArgs) * size_t(nt));
  L->off_units = off;   off += align_up(sizeof(ft::BatchUnit) * size_t(max_units));
  L->off_final = off;   off += align_up(sizeof(BatchFinalDesc) * size_t(nt));
  L->off_partial = off; off += align_up(sizeof(float) * size_t(max_partial));
  L->off_errpart = off; off += align_up(sizeof(double) * 2 * size_t(L->grid_eval));
  L->total = off;
  L->max_units = max_units;
  L->max_partial_floats = max_partial;
  return FT_OK;
}

}  // namespace

struct ft_batch {
  ft_config cfg;
  int num_sms = 0;
  std::vector<TensorInfo> tensors;
  std::vector<ClassInfo> classes;
  Layout L;
  char *ws = nullptr;
  cudaStream_t capture = nullptr;
  // per-class streams and join events: each class's factor and core passes
  // form one branch of the captured graph, all branches joining at finalize
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> joined;
  cudaEvent_t forked = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  int64_t graph_kernels = 0;
};

namespace {

template <typename T>
T *bws(ft_batch *b, size_t off) {
  return reinterpret_cast<T *>(b->ws + off);
}

// Units of every class for the classes' current unit sizes; the partial of
// each unit gets its own slot.  Uploads units and finalize descriptors.
ft_status layout_units(ft_batch *b, cudaStream_t st) {
  std::vector<ft::BatchUnit> units;
  std::vector<BatchFinalDesc> fin(b->tensors.size());
  int64_t poff = 0, elem = 0;
  for (ClassInfo &c : b->classes) {
    c.unit_first = int64_t(units.size());
    // units of each tensor (partials of a tensor in consecutive slots), then
    // dealt round-robin over the class's tensors: CTA b takes units b, b + G,
    // ..., so at any time the CTAs work on many tensors at once instead of
    // all on the rows of one
    std::vector<std::vector<ft::BatchUnit>> per;
    for (int t : c.tensors) {
      const TensorInfo &ti = b->tensors[size_t(t)];
      BatchFinalDesc &fd = fin[size_t(t)];
      memset(&fd, 0, sizeof(fd));
      fd.N = ti.N;
      fd.K = ti.K;
      fd.R = ti.R;
      for (int n = 0; n < ti.N; ++n) {
        fd.B[n] = ti.B[n];
        fd.J[n] = ti.J[n];
      }
      fd.inv_nnz = ti.nnz > 0 ? float(1.0 / double(ti.nnz)) : 0.f;
      fd.poff = poff;
      const int64_t pfl = 2LL * ti.N * ti.K * ti.K;
      const int64_t nu = std::max<int64_t>(1, (ti.ntiles + c.unit_tiles - 1) / c.unit_tiles);
      per.emplace_back();
      for (int64_t k = 0; k < nu; ++k) {
        ft::BatchUnit u;
        u.tensor = t;
        u.pad = 0;
        u.tile_begin = k * c.unit_tiles;
        u.tile_end = std::min<int64_t>(ti.ntiles, (k + 1) * c.unit_tiles);
        u.poff = poff;
        poff += pfl;
        per.back().push_back(u);
      }
      fd.nunits = int(nu);
    }
    for (size_t r = 0;; ++r) {
      bool any = false;
      for (const std::vector<ft::BatchUnit> &v : per)
        if (r < v.size()) {
          units.push_back(v[r]);
          any = true;
        }
      if (!any) break;
    }
    c.nunits = int64_t(units.size()) - c.unit_first;
  }
  // finalize index space in tensor order
  for (size_t t = 0; t < fin.size(); ++t) {
    fin[t].elem_begin = elem;
    elem += int64_t(fin[t].N) * fin[t].K * fin[t].K;
  }
  if (int64_t(units.size()) > b->L.max_units || poff > b->L.max_partial_floats) return FT_ERR_WORKSPACE;
  if (cudaMemcpyAsync(bws<ft::BatchUnit>(b, b->L.off_units), units.data(), sizeof(ft::BatchUnit) * units.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(bws<BatchFinalDesc>(b, b->L.off_final), fin.data(), sizeof(BatchFinalDesc) * fin.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FT_ERR_CUDA;
  return FT_OK;
}

ft::BatchArgs class_args(ft_batch *b, const ClassInfo &c) {
  ft::BatchArgs a;
  a.tensors = bws<ft::EpochArgs>(b, b->L.off_tensors);
  a.units = bws<ft::BatchUnit>(b, b->L.off_units) + c.unit_first;
  a.nunits = int(c.nunits);
  a.partial = bws<float>(b, b->L.off_partial);
  a.hyper = bws<float>(b, b->L.off_hyper);
  return a;
}

int class_grid(const ft_batch *b, const ClassInfo &c, bool core) {
  const int occ = core ? c.occ_core : c.occ_factor;
  const int bps = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, occ) : occ;
  const int64_t g = std::min<int64_t>(int64_t(b->num_sms) * bps, std::max<int64_t>(c.nunits, 1));
  return int(g);
}

cudaError_t launch_core(ft_batch *b, const ClassInfo &c, cudaStream_t st) {
  ft::BatchArgs a = class_args(b, c);
  void *argv[] = {&a};
  return cudaLaunchKernel(c.ks.batch_core, dim3(class_grid(b, c, true)), dim3(c.ks.batch_core_threads), argv,
                          c.ks.batch_core_smem, st);
}

// Capture factor passes, core passes and the finalize into one graph: the
// classes touch disjoint tensors, so each class's factor pass -> core pass
// is its own branch (concurrent with the other classes), and the finalize
// over every tensor waits for all branches.
ft_status capture(ft_batch *b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaStream_t st = b->capture;
  const size_t nc = b->classes.size();
  while (b->branch.size() < nc) {
    cudaStream_t s2 = nullptr;
    cudaEvent_t e2 = nullptr;
    if (cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) return FT_ERR_CUDA;
    b->branch.push_back(s2);
    if (cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) return FT_ERR_CUDA;
    b->joined.push_back(e2);
  }
  if (!b->forked && cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming) != cudaSuccess) return FT_ERR_CUDA;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FT_ERR_CUDA;
  bool ok = cudaEventRecord(b->forked, st) == cudaSuccess;
  int64_t kernels = 0;
  for (size_t k = 0; k < nc; ++k) {
    const ClassInfo &c = b->classes[k];
    cudaStream_t bs = b->branch[k];
    ok = ok && cudaStreamWaitEvent(bs, b->forked, 0) == cudaSuccess;
    ft::BatchArgs a = class_args(b, c);
    void *argv[] = {&a};
    ok = ok && cudaLaunchKernel(c.ks.batch_factor, dim3(class_grid(b, c, false)), dim3(c.ks.batch_factor_threads),
                                argv, c.ks.factor_smem, bs) == cudaSuccess;
    ok = ok && launch_core(b, c, bs) == cudaSuccess;
    ok = ok && cudaEventRecord(b->joined[k], bs) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(st, b->joined[k], 0) == cudaSuccess;
    kernels += 2;
  }
  int64_t total = 0;
  for (const TensorInfo &ti : b->tensors) total += int64_t(ti.N) * ti.K * ti.K;
  FinalArgs f;
  f.d = bws<BatchFinalDesc>(b, b->L.off_final);
  f.ntensors = int(b->tensors.size());
  f.total = total;
  f.partial = bws<float>(b, b->L.off_partial);
  f.hyper = bws<float>(b, b->L.off_hyper);
  void *fargv[] = {&f};
  ok = ok && cudaLaunchKernel(reinterpret_cast<const void *>(&k_batch_finalize), dim3(unsigned((total + 7) / 8)),
                              dim3(256), fargv, 0, st) == cudaSuccess;   // one warp per element
  ++kernels;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (!ok || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return FT_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return FT_ERR_CUDA;
  b->graph_kernels = kernels;
  return FT_OK;
}

}  // namespace

extern "C" {

ft_status ft_batch_workspace_size(int ntensors, const ft_tensor_desc *tensors, const ft_config *cfg,
                                  size_t *bytes) {
  if (!bytes) return FT_ERR_ARG;
  ft_config c;
  std::vector<TensorInfo> ts;
  std::vector<ClassInfo> cs;
  Layout L;
  int sms = 0;
  const ft_status s = plan_batch(ntensors, tensors, cfg, &c, &ts, &cs, &L, &sms);
  if (s != FT_OK) return s;
  *bytes = L.total;
  return FT_OK;
}

ft_status ft_batch_init(ft_batch **out, int ntensors, const ft_tensor_desc *tensors, const ft_config *cfg,
                        void *workspace, size_t ws_bytes, void *stream) {
  if (!out || !workspace) return FT_ERR_ARG;
  *out = nullptr;
  ft_batch *b = new (std::nothrow) ft_batch();
  if (!b) return FT_ERR_ARG;
  ft_status s = plan_batch(ntensors, tensors, cfg, &b->cfg, &b->tensors, &b->classes, &b->L, &b->num_sms);
  if (s != FT_OK) { delete b; return s; }
  if (ws_bytes < b->L.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) {
    delete b;
    return FT_ERR_WORKSPACE;
  }
  b->ws = static_cast<char *>(workspace);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *err = bws<int>(b, b->L.off_err);
  if (cudaMemsetAsync(b->ws, 0, b->L.off_tensors, st) != cudaSuccess) { delete b; return FT_ERR_CUDA; }
  // validate every tensor's coordinates and values
  for (const TensorInfo &ti : b->tensors) {
    if (ti.nnz == 0) continue;
    ValidateOne v;
    memset(&v, 0, sizeof(v));
    for (int n = 0; n < ti.N; ++n) {
      v.idx[n] = ti.idx[n];
      v.I[n] = ti.I[n];
    }
    v.N = ti.N;
    v.vals = ti.vals;
    v.nnz = ti.nnz;
    v.err = err;
    void *argv[] = {&v};
    const int grid = int(std::min<int64_t>((ti.nnz + 255) / 256, int64_t(b->num_sms) * 8));
    if (cudaLaunchKernel(reinterpret_cast<const void *>(&k_batch_validate), dim3(grid), dim3(256), argv, 0, st) !=
        cudaSuccess) {
      delete b;
      return FT_ERR_CUDA;
    }
    ++b->launches;
  }
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    delete b;
    return FT_ERR_CUDA;
  }
  if (h_err & ft::ERRBIT_INDEX) { delete b; return FT_ERR_INDEX; }
  if (h_err & ft::ERRBIT_VALUE) { delete b; return FT_ERR_NONFINITE; }
  // per-tensor arguments in the workspace
  std::vector<ft::EpochArgs> args(b->tensors.size());
  for (size_t t = 0; t < b->tensors.size(); ++t) {
    const TensorInfo &ti = b->tensors[t];
    ft::EpochArgs &a = args[t];
    memset(&a, 0, sizeof(a));
    int offJ = 0;
    for (int n = 0; n < ti.N; ++n) {
      a.idx[n] = ti.idx[n];
      a.A[n] = ti.A[n];
      a.B[n] = ti.B[n];
      a.I[n] = ti.I[n];
      a.J[n] = ti.J[n];
      a.offJ[n] = offJ;
      offJ += ti.J[n];
      if (ti.J[n] == ti.K && (reinterpret_cast<uintptr_t>(ti.A[n]) % 16) == 0) a.vecmask |= 1u << n;
      if (ti.J[n] % 4 == 0 && (reinterpret_cast<uintptr_t>(ti.A[n]) % 16) == 0) a.vec4mask |= 1u << n;
    }
    a.sumJ = offJ;
    a.R = ti.R;
    a.vals = ti.vals;
    a.begin = 0;
    a.end = ti.nnz;
    a.err = err;
  }
  if (cudaMemcpyAsync(bws<ft::EpochArgs>(b, b->L.off_tensors), args.data(), sizeof(ft::EpochArgs) * args.size(),
                      cudaMemcpyHostToDevice, st) != cudaSuccess) {
    delete b;
    return FT_ERR_CUDA;
  }
  s = layout_units(b, st);
  if (s == FT_OK && cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) s = FT_ERR_CUDA;
  if (s == FT_OK) s = capture(b);
  if (s != FT_OK) {
    ft_batch_destroy(b);
    return s;
  }
  *out = b;
  return FT_OK;
}

ft_status ft_batch_tune(ft_batch *b, void *stream) {
  if (!b) return FT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return FT_ERR_CUDA; }
  ft_status s = FT_OK;
  for (ClassInfo &c : b->classes) {
    float best = 1e30f;
    int best_u = c.unit_tiles, best_b = c.ctas_per_sm;
    std::vector<int> bps_cands = {0};
    for (int v = 1; v < c.occ_core; ++v) bps_cands.push_back(v);
    for (int ut : kUnitTiles) {
      for (int bps : bps_cands) {
        c.unit_tiles = ut;
        c.ctas_per_sm = bps;
        s = layout_units(b, st);
        if (s != FT_OK) break;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && s == FT_OK; ++rep) {  // the second run is timed
          if (cudaEventRecord(e0, st) != cudaSuccess || launch_core(b, c, st) != cudaSuccess ||
              cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            s = FT_ERR_CUDA;
          ++b->launches;
        }
        if (s != FT_OK) break;
        if (ms < best) {
          best = ms;
          best_u = ut;
          best_b = bps;
        }
      }
      if (s != FT_OK) break;
    }
    c.unit_tiles = best_u;
    c.ctas_per_sm = best_b;
    if (s != FT_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != FT_OK) return s;
  s = layout_units(b, st);
  if (s != FT_OK) return s;
  return capture(b);
}

ft_status ft_batch_epoch(ft_batch *b, float lr_a, float lambda_a, float lr_b, float lambda_b, void *stream) {
  if (!b || !b->exec) return FT_ERR_ARG;
  if (!std::isfinite(lr_a) || !std::isfinite(lambda_a) || !std::isfinite(lr_b) || !std::isfinite(lambda_b))
    return FT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_set_hyper<<<1, 32, 0, st>>>(bws<float>(b, b->L.off_hyper), lr_a, lambda_a, lr_b, lambda_b);
  if (cudaGetLastError() != cudaSuccess) return FT_ERR_CUDA;
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return FT_ERR_CUDA;
  b->launches += 1 + b->graph_kernels;
  return FT_OK;
}

ft_status ft_batch_rmse(ft_batch *b, int tensor, int64_t n, const int32_t *const *idx, const float *vals,
                        double *out3, void *stream) {
  if (!b || !out3 || tensor < 0 || tensor >= int(b->tensors.size())) return FT_ERR_ARG;
  if (n < 0 || n > INT32_MAX || (n > 0 && (!idx || !vals))) return FT_ERR_ARG;
  const TensorInfo &ti = b->tensors[size_t(tensor)];
  ft::EvalSet es;
  if (!(ti.K == 16 ? ft_eval_16(ti.N, &es) : ft_eval_32(ti.N, &es))) return FT_ERR_SHAPE;
  const int occ = occupancy(es.errors, 256, es.smem);
  if (occ < 1) return FT_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ft::EpochArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < ti.N; ++k) {
    if (n > 0 && !idx[k]) return FT_ERR_ARG;
    a.idx[k] = n > 0 ? idx[k] : nullptr;
    a.A[k] = ti.A[k];
    a.B[k] = ti.B[k];
    a.I[k] = ti.I[k];
    a.J[k] = ti.J[k];
    if (ti.J[k] == ti.K && (reinterpret_cast<uintptr_t>(ti.A[k]) % 16) == 0) a.vecmask |= 1u << k;
    if (ti.J[k] % 4 == 0 && (reinterpret_cast<uintptr_t>(ti.A[k]) % 16) == 0) a.vec4mask |= 1u << k;
  }
  a.R = ti.R;
  a.vals = vals;
  a.begin = 0;
  a.end = n;
  int *err = bws<int>(b, b->L.off_err);
  a.err = err;
  a.err_partial = bws<double>(b, b->L.off_errpart);
  const int grid = std::min(b->L.grid_eval, b->num_sms * occ);
  void *argv[] = {&a};
  if (cudaLaunchKernel(es.errors, dim3(grid), dim3(256), argv, es.smem, st) != cudaSuccess) return FT_ERR_CUDA;
  ErrFinal f;
  f.part = a.err_partial;
  f.nparts = grid;
  f.n = n;
  f.out3 = reinterpret_cast<double *>(reinterpret_cast<char *>(err) + 64);
  void *fargv[] = {&f};
  if (cudaLaunchKernel(reinterpret_cast<const void *>(&k_batch_errors_final), dim3(1), dim3(32), fargv, 0, st) !=
      cudaSuccess)
    return FT_ERR_CUDA;
  b->launches += 2;
  int h_err = 0;
  if (cudaMemcpyAsync(out3, f.out3, sizeof(double) * 3, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FT_ERR_CUDA;
  if (h_err) {
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return FT_ERR_CUDA;
    return (h_err & ft::ERRBIT_INDEX) ? FT_ERR_INDEX : FT_ERR_NONFINITE;
  }
  return FT_OK;
}

int ft_batch_num_classes(const ft_batch *b) { return b ? int(b->classes.size()) : 0; }

ft_status ft_batch_class_info(const ft_batch *b, int cls, int64_t *out6) {
  if (!b || !out6 || cls < 0 || cls >= int(b->classes.size())) return FT_ERR_ARG;
  const ClassInfo &c = b->classes[size_t(cls)];
  out6[0] = c.N;
  out6[1] = c.K;
  out6[2] = int64_t(c.tensors.size());
  out6[3] = c.unit_tiles;
  out6[4] = c.ctas_per_sm > 0 ? c.ctas_per_sm : c.occ_core;
  out6[5] = c.nunits;
  return FT_OK;
}

int64_t ft_batch_launch_count(const ft_batch *b) { return b ? b->launches : 0; }

void ft_batch_destroy(ft_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s2 : b->branch) cudaStreamDestroy(s2);
  for (cudaEvent_t e2 : b->joined) cudaEventDestroy(e2);
  if (b->forked) cudaEventDestroy(b->forked);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

}  // extern "C"
