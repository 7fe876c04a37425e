// C-ABI runtime of libqs: sim lifetime, device workspace, host-side
// validation, staging of host inputs, layout switching between the
// column-major (gates) and row-major (measurement) tableau, the op log that
// qs_sim_sample replays, and tableau export. Declarations and the contract of
// every entry point are in include/qs.h.
//
// Control flow follows Alg. 2 of the paper (Sec. 4.1): windows of gates are
// applied with one kernel each; a measurement window first switches the
// tableau to row-major (Alg. 4) and then runs the measurements in order. The
// layout switch is lazy: each layout is rebuilt only when the other one has
// been modified since.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qs_internal.cuh"

using namespace qs;

namespace {

thread_local std::string g_last_error;

// NVTX range over one ABI call (shows in Nsight timelines; no cost without a tool)
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

struct Op {
  enum Kind { kHostLayer, kDevLayers, kHostMeasure, kDevMeasure, kNoise } kind;
  std::vector<uint32_t> packed;  // kHostLayer: 2 words per gate
  const uint32_t *dev = nullptr; // kDevLayers: packed gates; kDevMeasure: qubit list
  std::vector<int64_t> ptr;      // kDevLayers: offsets of the replayed layers (+1)
  std::vector<uint32_t> qubits;  // kHostMeasure; kNoise: targets
  uint32_t count = 0;            // kDevMeasure
  uint64_t m0 = 0;               // first record index of a measurement op
  int noise_kind = 0;            // kNoise: QS_NOISE_*
  uint64_t thr = 0;              // kNoise: a shot fires iff its 32-bit draw u < thr
  uint64_t ordinal = 0;          // kNoise: index among the noise ops (the draw's e)
  uint64_t dev_off = 0;          // kNoise: offset of its targets in the sim's noise buffer (words)
};

constexpr int kRing = 4;
constexpr uint32_t kBlockedMinCount = 16;    // windows this long use blocked measurement
constexpr uint32_t kBlockedMinQubits = 64;
constexpr uint32_t kMaxQubits = 1u << 20;
// Frame layers cover a qubit's shot words in chunks of 512 words along grid.y
// (at most 65,535): 2e9 shots are 31.25 M words, 61,036 chunks.
constexpr uint64_t kMaxShots = 2000000000ull;

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

struct Plan {
  size_t X, Z, RX, RZ, S, colx, mst, detx, detz, dets, err, record, kinds, stage, blk, qsig, invp, total;
  uint64_t record_cap;
  size_t stage_bytes;
};

Plan make_plan(const Layout &L, const qs_options *opt) {
  Plan p;
  Carve c;
  p.record_cap = (opt && opt->record_capacity) ? opt->record_capacity : 16ull * L.n + 65536;
  p.stage_bytes = std::max<size_t>(8ull * (L.n + 64), 256 * 1024);
  const size_t colb = (size_t)L.ncols * L.cs * 8, rowb = (size_t)L.nrows * L.rs * 8;
  p.X = c.take(colb);
  p.Z = c.take(colb);
  p.RX = c.take(rowb);
  p.RZ = c.take(rowb);
  p.S = c.take((size_t)L.cs * 8);
  p.colx = c.take((size_t)L.cs * 8);
  p.mst = c.take(kMeasStateWords * 8);
  p.detx = c.take((size_t)kDetBlocks * L.rs * 8);
  p.detz = c.take((size_t)kDetBlocks * L.rs * 8);
  p.dets = c.take((size_t)kDetBlocks * 4);
  p.err = c.take(4);
  p.record = c.take(p.record_cap);
  p.kinds = c.take(p.record_cap);
  p.stage = c.take(p.stage_bytes);
  p.blk = c.take(blocked_scratch_bytes(L));
  const bool inverse = opt && (opt->flags & QS_FLAG_INVERSE_TABLEAU);
  p.qsig = c.take(inverse ? 2ull * L.rs * 8 : 0);
  p.invp = c.take(inverse ? inv_scratch_words(L) * 8 : 0);
  p.total = c.off;
  return p;
}

bool is_two(uint32_t t) { return t >= QS_CX && t <= QS_ISWAP; }

}  // namespace

struct qs_sim {
  Dev d{};
  Plan plan{};
  cudaStream_t stream = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  bool cols_valid = true, rows_valid = false;
  bool broken = false;
  uint64_t n_meas = 0;
  uint64_t n_noise = 0;
  uint8_t *dstage = nullptr;
  uint8_t *hstage[kRing] = {};
  cudaEvent_t ev[kRing] = {};
  int ring = 0;
  std::vector<Op> ops;
  std::vector<uint32_t> stamp;
  uint32_t stamp_id = 0;
  uint64_t launches = 0;
  uint32_t flags = 0;
  void *blk = nullptr;  // scratch of the blocked measurement
  bool resumed = false; // state restored by qs_sim_tableau_import: no op log from |0...0>
  std::unique_ptr<KernelTimer> timer;  // qs_sim_set_timing
  // every noise op's targets, uploaded once for qs_sim_sample's replays (valid
  // while noise_dev_ops equals n_noise; it grows, never shrinks, until destroy)
  uint32_t *noise_dev = nullptr;
  size_t noise_dev_words = 0;
  uint64_t noise_dev_ops = 0;
};

namespace {

int cuda_fail(qs_sim *s, cudaError_t e, const char *what) {
  if (s) s->broken = true;
  return fail(QS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define QS_CUDA(sim, call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(sim, e_, #call); \
  } while (0)

// Next pinned host slot, waiting until its previous copy has finished.
uint8_t *ring_slot(qs_sim *s, int *slot) {
  int i = s->ring;
  s->ring = (s->ring + 1) % kRing;
  if (cudaEventSynchronize(s->ev[i]) != cudaSuccess) return nullptr;
  *slot = i;
  return s->hstage[i];
}

// Copies `bytes` (<= stage_bytes) from a pinned slot to the device staging area.
int upload(qs_sim *s, int slot, size_t bytes) {
  QS_CUDA(s, cudaMemcpyAsync(s->dstage, s->hstage[slot], bytes, cudaMemcpyHostToDevice, s->stream));
  QS_CUDA(s, cudaEventRecord(s->ev[slot], s->stream));
  return QS_OK;
}

int check_usable(qs_sim *s) {
  if (!s) return fail(QS_ERR_ARG, "sim is NULL");
  if (s->broken) return fail(QS_ERR_STATE, "sim is unusable after an earlier device error");
  return QS_OK;
}

int ensure_cols(qs_sim *s) {
  if (!s->cols_valid) {
    tbegin(s->d.timer, QS_TIME_TRANSPOSE, s->stream);
    QS_CUDA(s, launch_to_cols(s->d, s->stream));
    tend(s->d.timer, QS_TIME_TRANSPOSE, s->stream);
    s->launches += 2;
    s->cols_valid = true;
  }
  return QS_OK;
}

int ensure_rows(qs_sim *s) {
  if (!s->rows_valid) {
    tbegin(s->d.timer, QS_TIME_TRANSPOSE, s->stream);
    QS_CUDA(s, launch_to_rows(s->d, s->stream));
    tend(s->d.timer, QS_TIME_TRANSPOSE, s->stream);
    s->launches += 2;
    s->rows_valid = true;
  }
  return QS_OK;
}

// Validates one layer; packs into out (2 words per gate). Returns QS_OK or QS_ERR_ARG.
int validate_pack(uint32_t n, const qs_gate *g, size_t count, std::vector<uint32_t> &stamp,
                  uint32_t &stamp_id, uint32_t *out, const char *where) {
  if (stamp.size() < n) stamp.assign(n, 0);
  if (++stamp_id == 0) {
    std::fill(stamp.begin(), stamp.end(), 0);
    stamp_id = 1;
  }
  char buf[160];
  for (size_t i = 0; i < count; ++i) {
    const uint32_t t = g[i].type, a = g[i].q0, b = g[i].q1;
    if (t >= QS_NUM_GATE_TYPES) {
      snprintf(buf, sizeof buf, "%s gate %zu: unknown gate type %u", where, i, t);
      return fail(QS_ERR_ARG, buf);
    }
    if (a >= n || (is_two(t) && b >= n)) {
      snprintf(buf, sizeof buf, "%s gate %zu: qubit out of range (n = %u)", where, i, n);
      return fail(QS_ERR_ARG, buf);
    }
    if (is_two(t) && a == b) {
      snprintf(buf, sizeof buf, "%s gate %zu: two-qubit gate on one qubit %u", where, i, a);
      return fail(QS_ERR_ARG, buf);
    }
    if (stamp[a] == stamp_id || (is_two(t) && stamp[b] == stamp_id)) {
      snprintf(buf, sizeof buf, "%s gate %zu: qubit used twice in one layer", where, i);
      return fail(QS_ERR_ARG, buf);
    }
    stamp[a] = stamp_id;
    if (is_two(t)) stamp[b] = stamp_id;
    out[2 * i] = (t << 24) | a;
    out[2 * i + 1] = is_two(t) ? b : 0;
  }
  return QS_OK;
}

// Enqueues layers [0, ptr.size() - 1) given by absolute gate offsets `ptr`
// of device gate records `packed` on the tableau (S != nullptr) or on frames.
// Runs of layers go through the fused shared-memory kernel when the word slice
// fits, else one kernel per layer.
int run_dev_layers(qs_sim *s, uint64_t *X, uint64_t *Z, uint64_t *S, uint32_t stride,
                   const uint32_t *packed, const int64_t *ptr, size_t nlayers, bool tableau) {
  const uint32_t n = s->d.L.n;
  if (nlayers == 0) return QS_OK;
  if (fused_fits(n) && !(s->flags & QS_FLAG_NO_FUSION) && !(tableau && s->d.inverse)) {
    const size_t cap = s->plan.stage_bytes / 8 - 1;  // layers per staged offset table
    for (size_t l0 = 0; l0 < nlayers; l0 += cap) {
      const size_t L = std::min(cap, nlayers - l0);
      int slot;
      uint8_t *h = ring_slot(s, &slot);
      if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
      memcpy(h, ptr + l0, (L + 1) * 8);
      int rc = upload(s, slot, (L + 1) * 8);
      if (rc) return rc;
      int64_t max_gates = 0;  // layers hold at most n gates (checked when they were added)
      for (size_t l = l0; l < l0 + L; ++l) max_gates = std::max<int64_t>(max_gates, ptr[l + 1] - ptr[l]);
      QS_CUDA(s, launch_fused_segment(X, Z, S, n, stride, stride, packed,
                                      reinterpret_cast<const int64_t *>(s->dstage), (uint32_t)L,
                                      (uint32_t)max_gates, s->d.err, s->stream));
      s->launches += 1;
    }
    return QS_OK;
  }
  for (size_t l = 0; l < nlayers; ++l) {
    const int64_t a = ptr[l], cnt = ptr[l + 1] - a;
    if (cnt == 0) continue;
    if (tableau && s->d.inverse)
      QS_CUDA(s, launch_inv_gate_layer(s->d, packed + 2 * a, (uint32_t)cnt, s->stream));
    else if (tableau)
      QS_CUDA(s, launch_gate_layer(s->d, packed + 2 * a, (uint32_t)cnt, s->stream));
    else
      QS_CUDA(s, launch_frame_layer(X, Z, n, stride, packed + 2 * a, (uint32_t)cnt, s->d.err,
                                    s->stream));
    s->launches += 1;
  }
  return QS_OK;
}

}  // namespace

// device address of the allocation-free sampler's static array on the current
// device (looked up once per device; defined with the array further below)
static cudaError_t noalloc_setup(void **addr);

extern "C" {

const char *qs_version(void) { return "qs-gb300 0.1 (sm_103a)"; }

const char *qs_last_error(void) { return g_last_error.c_str(); }

size_t qs_sim_required_bytes(uint32_t n, const qs_options *opt) {
  if (n == 0 || n > kMaxQubits) return 0;
  return make_plan(make_layout(n), opt).total;
}

int qs_sim_create(uint32_t n, const qs_options *opt, void *cuda_stream, void *workspace,
                  size_t workspace_bytes, qs_sim **out) {
  if (!out) return fail(QS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n == 0 || n > kMaxQubits) return fail(QS_ERR_ARG, "n must be in [1, 2^20]");
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(QS_ERR_ARG, "workspace must be 256-byte aligned");
  qs_sim *s = new (std::nothrow) qs_sim();
  if (!s) return fail(QS_ERR_OOM, "host allocation failed");
  s->d.L = make_layout(n);
  s->plan = make_plan(s->d.L, opt);
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->flags = opt ? opt->flags : 0u;
  s->d.wide_offsets = (s->flags & QS_FLAG_WIDE_OFFSETS) != 0;
  s->d.step_symbolic = (s->flags & QS_FLAG_STEP_SYMBOLIC) != 0;
  s->d.inverse = (s->flags & QS_FLAG_INVERSE_TABLEAU) != 0;
  if (workspace) {
    if (workspace_bytes < s->plan.total) {
      delete s;
      return fail(QS_ERR_SIZE, "workspace smaller than qs_sim_required_bytes");
    }
    s->ws = workspace;
  } else {
    cudaError_t e = cudaMalloc(&s->ws, s->plan.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return fail(QS_ERR_OOM, std::string("cudaMalloc of the tableau failed: ") + cudaGetErrorString(e));
    }
    s->owns_ws = true;
  }
  s->ws_bytes = s->plan.total;
  uint8_t *b = static_cast<uint8_t *>(s->ws);
  const Plan &p = s->plan;
  s->d.X = reinterpret_cast<uint64_t *>(b + p.X);
  s->d.Z = reinterpret_cast<uint64_t *>(b + p.Z);
  s->d.RX = reinterpret_cast<uint64_t *>(b + p.RX);
  s->d.RZ = reinterpret_cast<uint64_t *>(b + p.RZ);
  s->d.S = reinterpret_cast<uint64_t *>(b + p.S);
  s->d.colx = reinterpret_cast<uint32_t *>(b + p.colx);
  s->d.mst = reinterpret_cast<int64_t *>(b + p.mst);
  s->d.det_x = reinterpret_cast<uint64_t *>(b + p.detx);
  s->d.det_z = reinterpret_cast<uint64_t *>(b + p.detz);
  s->d.det_scal = reinterpret_cast<int32_t *>(b + p.dets);
  s->d.err = reinterpret_cast<uint32_t *>(b + p.err);
  s->d.record = b + p.record;
  s->d.kinds = b + p.kinds;
  s->d.record_cap = p.record_cap;
  s->dstage = b + p.stage;
  s->blk = b + p.blk;
  s->d.qsig = s->d.inverse ? reinterpret_cast<uint64_t *>(b + p.qsig) : nullptr;
  s->d.inv_part = s->d.inverse ? reinterpret_cast<uint64_t *>(b + p.invp) : nullptr;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    // place the allocation-free sampler's array on this device now, before the
    // caller may reserve the rest of the GPU; a failure here only matters to
    // qs_sim_sample_noalloc, which retries and reports it
    void *unused = nullptr;
    if (noalloc_setup(&unused) != cudaSuccess) cudaGetLastError();
  }
  s->d.sms = 152;
  cudaDeviceGetAttribute(&s->d.sms, cudaDevAttrMultiProcessorCount, dev);
  for (int i = 0; i < kRing; ++i) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&s->hstage[i]), p.stage_bytes,
                                  cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      qs_sim_destroy(s);
      return fail(QS_ERR_OOM, std::string("pinned staging allocation failed: ") + cudaGetErrorString(e));
    }
  }
  int rc = qs_sim_reset(s, nullptr);
  if (rc != QS_OK) {
    std::string msg = g_last_error;
    qs_sim_destroy(s);
    return fail(rc, msg);
  }
  *out = s;
  return QS_OK;
}

int qs_sim_destroy(qs_sim *s) {
  if (!s) return QS_OK;
  cudaStreamSynchronize(s->stream);
  for (int i = 0; i < kRing; ++i) {
    if (s->ev[i]) cudaEventDestroy(s->ev[i]);
    if (s->hstage[i]) cudaFreeHost(s->hstage[i]);
  }
  if (s->owns_ws && s->ws) cudaFree(s->ws);
  if (s->noise_dev) cudaFree(s->noise_dev);
  delete s;
  return QS_OK;
}

int qs_sim_reset(qs_sim *s, const uint8_t *initstate) {
  int rc = check_usable(s);
  if (rc) return rc;
  const uint32_t n = s->d.L.n;
  const uint8_t *init_dev = nullptr;
  if (initstate) {
    int slot;
    uint8_t *h = ring_slot(s, &slot);
    if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
    for (uint32_t i = 0; i < n; ++i) h[i] = initstate[i] ? 1 : 0;
    if ((rc = upload(s, slot, n))) return rc;
    init_dev = s->dstage;
  }
  QS_CUDA(s, cudaMemsetAsync(s->d.err, 0, 4, s->stream));
  if (s->d.inverse) {
    // same bits as the CHP mode, no per-row signs; the basis state sits in S_S
    QS_CUDA(s, launch_init(s->d, nullptr, s->stream));
    QS_CUDA(s, launch_inv_init_signs(s->d, init_dev, s->stream));
    s->launches += 1;
  } else {
    QS_CUDA(s, launch_init(s->d, init_dev, s->stream));
  }
  QS_CUDA(s, launch_reset_meas_state(s->d, s->stream));
  s->launches += 3;
  s->cols_valid = true;
  s->rows_valid = false;
  s->n_meas = 0;
  s->n_noise = 0;
  s->ops.clear();
  s->resumed = false;
  s->noise_dev_ops = 0;  // the buffer is kept for the next program's noise ops
  return QS_OK;
}

int qs_sim_apply_layer(qs_sim *s, const qs_gate *gates, uint32_t n_gates) {
  Range range_("qs_sim_apply_layer");
  int rc = check_usable(s);
  if (rc) return rc;
  if (n_gates && !gates) return fail(QS_ERR_ARG, "gates is NULL");
  if (n_gates > s->d.L.n) return fail(QS_ERR_ARG, "more gates than qubits in one layer");
  Op op;
  op.kind = Op::kHostLayer;
  op.packed.resize(2 * (size_t)n_gates);
  if ((rc = validate_pack(s->d.L.n, gates, n_gates, s->stamp, s->stamp_id, op.packed.data(),
                          "layer")))
    return rc;
  if (n_gates == 0) return QS_OK;
  if ((rc = ensure_cols(s))) return rc;
  int slot;
  uint8_t *h = ring_slot(s, &slot);
  if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
  memcpy(h, op.packed.data(), op.packed.size() * 4);
  if ((rc = upload(s, slot, op.packed.size() * 4))) return rc;
  tbegin(s->d.timer, QS_TIME_GATES, s->stream);
  if (s->d.inverse)
    QS_CUDA(s, launch_inv_gate_layer(s->d, reinterpret_cast<const uint32_t *>(s->dstage), n_gates,
                                     s->stream));
  else
    QS_CUDA(s, launch_gate_layer(s->d, reinterpret_cast<const uint32_t *>(s->dstage), n_gates,
                                 s->stream));
  tend(s->d.timer, QS_TIME_GATES, s->stream);
  s->launches += 1;
  s->rows_valid = false;
  s->ops.push_back(std::move(op));
  return QS_OK;
}

int qs_pack_layers(uint32_t n, const qs_gate *gates, const int64_t *layer_ptr, uint32_t n_layers,
                   uint32_t *packed) {
  if (n == 0 || n > kMaxQubits) return fail(QS_ERR_ARG, "n must be in [1, 2^20]");
  if (!layer_ptr || (n_layers && (!gates && layer_ptr[n_layers] > 0)) || !packed)
    return fail(QS_ERR_ARG, "NULL argument");
  if (layer_ptr[0] != 0) return fail(QS_ERR_ARG, "layer_ptr[0] must be 0");
  std::vector<uint32_t> stamp;
  uint32_t sid = 0;
  for (uint32_t l = 0; l < n_layers; ++l) {
    const int64_t a = layer_ptr[l], b = layer_ptr[l + 1];
    if (b < a) return fail(QS_ERR_ARG, "layer_ptr must be nondecreasing");
    if (b - a > (int64_t)n) return fail(QS_ERR_ARG, "more gates than qubits in one layer");
    char where[48];
    snprintf(where, sizeof where, "layer %u", l);
    int rc = validate_pack(n, gates + a, (size_t)(b - a), stamp, sid, packed + 2 * a, where);
    if (rc) return rc;
  }
  return QS_OK;
}

int qs_sim_apply_layers_dev(qs_sim *s, const uint32_t *packed_dev, const int64_t *layer_ptr,
                            uint32_t l_begin, uint32_t l_end) {
  Range range_("qs_sim_apply_layers_dev");
  int rc = check_usable(s);
  if (rc) return rc;
  if (!packed_dev || !layer_ptr) return fail(QS_ERR_ARG, "NULL argument");
  if (l_end < l_begin) return fail(QS_ERR_ARG, "l_end < l_begin");
  if (l_end == l_begin) return QS_OK;
  if ((rc = ensure_cols(s))) return rc;
  Op op;
  op.kind = Op::kDevLayers;
  op.dev = packed_dev;
  op.ptr.assign(layer_ptr + l_begin, layer_ptr + l_end + 1);
  if (op.ptr[0] < 0) return fail(QS_ERR_ARG, "negative layer_ptr");
  for (size_t l = 0; l + 1 < op.ptr.size(); ++l) {
    const int64_t cnt = op.ptr[l + 1] - op.ptr[l];
    if (cnt < 0 || cnt > (int64_t)s->d.L.n) return fail(QS_ERR_ARG, "bad layer_ptr");
  }
  tbegin(s->d.timer, QS_TIME_GATES, s->stream);
  if ((rc = run_dev_layers(s, s->d.X, s->d.Z, s->d.S, s->d.L.cs, packed_dev, op.ptr.data(),
                           op.ptr.size() - 1, true)))
    return rc;
  tend(s->d.timer, QS_TIME_GATES, s->stream);
  s->rows_valid = false;
  s->ops.push_back(std::move(op));
  return QS_OK;
}

static int measure_staged(qs_sim *s, const uint32_t *qdev, uint32_t count, uint64_t m0, qs_key key) {
  if (s->d.inverse) {  // Alg. 1, one measurement after another
    tbegin(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
    for (uint32_t i = 0; i < count; ++i) {
      int l = 0;
      QS_CUDA(s, launch_inv_measure_one(s->d, qdev, i, m0 + i, key, s->stream, &l));
      s->launches += (uint64_t)l;
    }
    tend(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
    return QS_OK;
  }
  if (!(s->flags & (QS_FLAG_UNPIPELINED_MEASURE | QS_FLAG_NO_BLOCKED_MEASURE)) &&
      measure_window_supported(s->d.L) && count >= kBlockedMinCount && s->d.L.n >= kBlockedMinQubits) {
    // blocks of up to 64 measurements; a block stops before a deterministic
    // outcome, which then goes through the single-measurement path. After two
    // blocks in a row that stop at their first step (a run of deterministic
    // outcomes), the rest of the window takes the pipelined path.
    // Each block starts at the window position a device cursor holds and moves
    // it on, so rounds of several blocks go out before the host reads how far
    // they got: one round doubles (up to 8 blocks) while rounds finish, and
    // drops back to one block after a block stopped short.
    const uint32_t *cur = block_cursor(s->d.L, s->blk);
    QS_CUDA(s, set_block_cursor(s->d.L, s->blk, 0, s->stream));
    s->launches += 1;
    uint32_t i = 0, empty_rounds = 0, per_round = 1;
    while (i < count) {
      if (empty_rounds >= 2) {
        int l = 0;
        tbegin(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
        QS_CUDA(s, launch_measure_window(s->d, qdev + i, count - i, m0 + i, key, s->stream, &l));
        tend(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
        s->launches += (uint64_t)l;
        break;
      }
      Range block_range("blocked measurement round");
      const uint32_t nb = std::min<uint32_t>(per_round, (count - i + 63) / 64);
      for (uint32_t b = 0; b < nb; ++b) {
        int l = 0;
        QS_CUDA(s, launch_measure_block(s->d, s->blk, qdev, count, m0, key, s->stream, &l));
        s->launches += (uint64_t)l;
      }
      uint32_t at = 0;
      QS_CUDA(s, cudaMemcpyAsync(&at, cur, 4, cudaMemcpyDeviceToHost, s->stream));
      QS_CUDA(s, cudaStreamSynchronize(s->stream));
      if (s->timer) s->timer->resolve();
      if (at < i || at > count) return fail(QS_ERR_INTERNAL, "blocked measurement cursor");
      const uint32_t done = at - i;
      i = at;
      if (i < count && done < 64 * nb) {
        // a block stopped before a deterministic outcome (the blocks after it
        // in the round did nothing): measure it alone and step past it
        int l = 0;
        tbegin(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
        QS_CUDA(s, launch_measure_window(s->d, qdev + i, 1, m0 + i, key, s->stream, &l));
        tend(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
        s->launches += (uint64_t)l;
        i += 1;
        QS_CUDA(s, set_block_cursor(s->d.L, s->blk, i, s->stream));
        s->launches += 1;
        empty_rounds = done == 0 ? empty_rounds + 1 : 0;
        per_round = 1;
      } else {
        empty_rounds = 0;
        per_round = std::min<uint32_t>(8, 2 * per_round);
      }
    }
    return QS_OK;
  }
  tbegin(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
  if (!(s->flags & QS_FLAG_UNPIPELINED_MEASURE) && measure_window_supported(s->d.L)) {
    int l = 0;
    QS_CUDA(s, launch_measure_window(s->d, qdev, count, m0, key, s->stream, &l));
    s->launches += (uint64_t)l;
  } else {
    for (uint32_t i = 0; i < count; ++i) {
      int l = 0;
      QS_CUDA(s, launch_measure_one(s->d, qdev, i, m0 + i, key, s->stream, &l));
      s->launches += (uint64_t)l;
    }
  }
  tend(s->d.timer, QS_TIME_MEASURE_SINGLE, s->stream);
  return QS_OK;
}

int qs_sim_measure(qs_sim *s, const uint32_t *qubits, uint32_t count, qs_key key,
                   uint8_t *outcomes) {
  Range range_("qs_sim_measure");
  int rc = check_usable(s);
  if (rc) return rc;
  if (count && !qubits) return fail(QS_ERR_ARG, "qubits is NULL");
  for (uint32_t i = 0; i < count; ++i)
    if (qubits[i] >= s->d.L.n) {
      char buf[96];
      snprintf(buf, sizeof buf, "measured qubit %u out of range (n = %u)", qubits[i], s->d.L.n);
      return fail(QS_ERR_ARG, buf);
    }
  if (s->n_meas + count > s->d.record_cap)
    return fail(QS_ERR_SIZE, "record capacity exceeded (qs_options.record_capacity)");
  if (count == 0) return QS_OK;
  if ((rc = ensure_rows(s))) return rc;
  const uint64_t m0 = s->n_meas;
  const uint32_t chunk = (uint32_t)(s->plan.stage_bytes / 4);
  for (uint32_t off = 0; off < count; off += chunk) {
    const uint32_t c = std::min(chunk, count - off);
    int slot;
    uint8_t *h = ring_slot(s, &slot);
    if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
    memcpy(h, qubits + off, (size_t)c * 4);
    if ((rc = upload(s, slot, (size_t)c * 4))) return rc;
    if ((rc = measure_staged(s, reinterpret_cast<const uint32_t *>(s->dstage), c, m0 + off, key)))
      return rc;
  }
  s->n_meas += count;
  s->cols_valid = false;
  Op op;
  op.kind = Op::kHostMeasure;
  op.qubits.assign(qubits, qubits + count);
  op.m0 = m0;
  s->ops.push_back(std::move(op));
  if (outcomes) {
    QS_CUDA(s, cudaMemcpyAsync(outcomes, s->d.record + m0, count, cudaMemcpyDeviceToHost, s->stream));
    return qs_sim_sync(s);
  }
  return QS_OK;
}

int qs_sim_measure_dev(qs_sim *s, const uint32_t *qubits_dev, uint32_t count, qs_key key) {
  Range range_("qs_sim_measure_dev");
  int rc = check_usable(s);
  if (rc) return rc;
  if (count && !qubits_dev) return fail(QS_ERR_ARG, "qubits_dev is NULL");
  if (s->n_meas + count > s->d.record_cap)
    return fail(QS_ERR_SIZE, "record capacity exceeded (qs_options.record_capacity)");
  if (count == 0) return QS_OK;
  if ((rc = ensure_rows(s))) return rc;
  const uint64_t m0 = s->n_meas;
  if ((rc = measure_staged(s, qubits_dev, count, m0, key))) return rc;
  s->n_meas += count;
  s->cols_valid = false;
  Op op;
  op.kind = Op::kDevMeasure;
  op.dev = qubits_dev;
  op.count = count;
  op.m0 = m0;
  s->ops.push_back(std::move(op));
  return QS_OK;
}

int qs_sim_noise(qs_sim *s, int kind, double p, const uint32_t *targets, uint32_t count) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (kind < 0 || kind >= QS_NUM_NOISE_KINDS) return fail(QS_ERR_ARG, "unknown noise kind");
  if (!(p >= 0.0 && p <= 1.0)) return fail(QS_ERR_ARG, "noise probability outside [0, 1]");
  if (count && !targets) return fail(QS_ERR_ARG, "targets is NULL");
  if (kind == QS_NOISE_DEPOLARIZE2 && (count & 1u))
    return fail(QS_ERR_ARG, "DEPOLARIZE2 takes pairs of targets");
  const uint32_t n = s->d.L.n;
  if (s->stamp.size() < n) s->stamp.assign(n, 0);
  if (++s->stamp_id == 0) {
    std::fill(s->stamp.begin(), s->stamp.end(), 0);
    s->stamp_id = 1;
  }
  for (uint32_t i = 0; i < count; ++i) {
    if (targets[i] >= n) return fail(QS_ERR_ARG, "noise target " + std::to_string(targets[i]) + " >= n");
    if (s->stamp[targets[i]] == s->stamp_id)
      return fail(QS_ERR_ARG, "noise target " + std::to_string(targets[i]) + " repeated");
    s->stamp[targets[i]] = s->stamp_id;
  }
  Op op;
  op.kind = Op::kNoise;
  op.noise_kind = kind;
  op.qubits.assign(targets, targets + count);
  // floor(p * 2^32) (multiplying by a power of two is exact); 2^32 fires always
  op.thr = p >= 1.0 ? 4294967296ull : (p > 0.0 ? (uint64_t)(p * 4294967296.0) : 0);
  op.ordinal = s->n_noise++;
  s->ops.push_back(std::move(op));
  return QS_OK;
}

uint64_t qs_sim_num_measurements(const qs_sim *s) { return s ? s->n_meas : 0; }

uint64_t qs_sim_launch_count(const qs_sim *s) { return s ? s->launches : 0; }

int qs_sim_set_timing(qs_sim *s, int on) {
  int rc = check_usable(s);
  if (rc) return rc;
  QS_CUDA(s, cudaStreamSynchronize(s->stream));
  if (!on) {
    s->d.timer = nullptr;
    s->timer.reset();
    return QS_OK;
  }
  if (!s->timer) {
    s->timer.reset(new (std::nothrow) KernelTimer());
    if (!s->timer) return fail(QS_ERR_OOM, "host allocation failed");
  }
  s->timer->clear();
  s->d.timer = s->timer.get();
  return QS_OK;
}

int qs_sim_timing(qs_sim *s, double *ms, uint64_t *count, uint32_t kinds) {
  if (!s) return fail(QS_ERR_ARG, "sim is NULL");
  if (!s->timer) return fail(QS_ERR_STATE, "timing is off (qs_sim_set_timing)");
  QS_CUDA(s, cudaStreamSynchronize(s->stream));
  s->timer->resolve();
  for (uint32_t k = 0; k < kinds && k < (uint32_t)QS_NUM_TIME_KINDS; ++k) {
    if (ms) ms[k] = s->timer->ms[k];
    if (count) count[k] = s->timer->count[k];
  }
  return QS_OK;
}

int qs_sim_record(qs_sim *s, uint64_t first, uint64_t count, uint8_t *dst) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (first > s->n_meas || count > s->n_meas - first)
    return fail(QS_ERR_ARG, "record range beyond the measurements");
  if (count && !dst) return fail(QS_ERR_ARG, "dst is NULL");
  if (count)
    QS_CUDA(s, cudaMemcpyAsync(dst, s->d.record + first, count, cudaMemcpyDeviceToHost, s->stream));
  return qs_sim_sync(s);
}

int qs_sim_record_kinds(qs_sim *s, uint64_t first, uint64_t count, uint8_t *dst) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (first > s->n_meas || count > s->n_meas - first)
    return fail(QS_ERR_ARG, "record range beyond the measurements");
  if (count && !dst) return fail(QS_ERR_ARG, "dst is NULL");
  if (count)
    QS_CUDA(s, cudaMemcpyAsync(dst, s->d.kinds + first, count, cudaMemcpyDeviceToHost, s->stream));
  return qs_sim_sync(s);
}

int qs_sim_sync(qs_sim *s) {
  if (!s) return fail(QS_ERR_ARG, "sim is NULL");
  if (s->broken) return fail(QS_ERR_STATE, "sim is unusable after an earlier device error");
  QS_CUDA(s, cudaStreamSynchronize(s->stream));
  uint32_t flags = 0;
  QS_CUDA(s, cudaMemcpy(&flags, s->d.err, 4, cudaMemcpyDeviceToHost));
  if (flags & kErrTimeout) {
    s->broken = true;
    return fail(QS_ERR_TIMEOUT, "a bounded device wait ran out");
  }
  if (flags) {
    s->broken = true;
    char buf[128];
    snprintf(buf, sizeof buf, "device self-check failed (flags 0x%x: odd phase=1, det=2, gate=4, qubit=8)",
             flags);
    return fail(QS_ERR_INTERNAL, buf);
  }
  return QS_OK;
}

// Replays a noise op on the frames: targets staged through the pinned ring in
// chunks (whole pairs for DEPOLARIZE2), target index continued across chunks.
static int replay_noise(qs_sim *s, const Op &op, uint64_t *FX, uint64_t *FZ, uint32_t fw, uint32_t ow,
                        uint64_t seed) {
  const bool pairs = op.noise_kind == QS_NOISE_DEPOLARIZE2;
  const uint32_t per = pairs ? 2 : 1;
  const uint32_t total = (uint32_t)op.qubits.size() / per;  // targets or pairs
  const uint32_t chunk = (uint32_t)(s->plan.stage_bytes / 4 / per);
  for (uint32_t t0 = 0; t0 < total; t0 += chunk) {
    const uint32_t c = std::min(chunk, total - t0);
    int slot;
    uint8_t *h = ring_slot(s, &slot);
    if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
    memcpy(h, op.qubits.data() + (size_t)t0 * per, (size_t)c * per * 4);
    int rc = upload(s, slot, (size_t)c * per * 4);
    if (rc) return rc;
    QS_CUDA(s, launch_frame_noise(FX, FZ, fw, ow, reinterpret_cast<uint32_t *>(s->dstage), c, t0,
                                  op.noise_kind, op.thr, op.ordinal, seed, s->stream));
    if (op.thr) s->launches += 1;
  }
  return QS_OK;
}

// Uploads the targets of every noise op of the op log into one device buffer
// (once per change of the op log), so that replays launch straight from it.
static int upload_noise_targets(qs_sim *s) {
  if (s->n_noise == 0 || s->noise_dev_ops == s->n_noise) return QS_OK;
  size_t words = 0;
  for (const Op &op : s->ops)
    if (op.kind == Op::kNoise) words += op.qubits.size();
  std::vector<uint32_t> host(std::max<size_t>(words, 1));
  size_t off = 0;
  for (Op &op : s->ops)
    if (op.kind == Op::kNoise) {
      op.dev_off = off;
      if (!op.qubits.empty()) memcpy(host.data() + off, op.qubits.data(), op.qubits.size() * 4);
      off += op.qubits.size();
    }
  if (words > s->noise_dev_words) {
    if (s->noise_dev) {
      QS_CUDA(s, cudaStreamSynchronize(s->stream));  // earlier replays may still read it
      QS_CUDA(s, cudaFree(s->noise_dev));
      s->noise_dev = nullptr;
      s->noise_dev_words = 0;
    }
    cudaError_t e = cudaMalloc(&s->noise_dev, words * 4);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s->noise_dev = nullptr;
      return fail(QS_ERR_OOM, "device buffer of the noise targets");
    }
    s->noise_dev_words = words;
  }
  QS_CUDA(s, cudaMemcpyAsync(s->noise_dev, host.data(), words * 4, cudaMemcpyHostToDevice, s->stream));
  QS_CUDA(s, cudaStreamSynchronize(s->stream));  // the host copy goes out of scope
  s->noise_dev_ops = s->n_noise;
  return QS_OK;
}

// One noise op straight from the uploaded targets.
static int replay_noise_dev(qs_sim *s, const Op &op, uint64_t *FX, uint64_t *FZ, uint32_t fw, uint32_t ow,
                            uint64_t seed) {
  const uint32_t per = op.noise_kind == QS_NOISE_DEPOLARIZE2 ? 2 : 1;
  const uint32_t total = (uint32_t)op.qubits.size() / per;
  QS_CUDA(s, launch_frame_noise(FX, FZ, fw, ow, s->noise_dev + op.dev_off, total, 0, op.noise_kind, op.thr,
                                op.ordinal, seed, s->stream));
  if (op.thr && total) s->launches += 1;
  return QS_OK;
}

static size_t sample_bytes(const qs_sim *s, uint64_t shots, uint64_t *fw_out, uint64_t *ow_out) {
  const uint64_t ow = (shots + 63) / 64;
  const uint64_t fw = (ow + 3) / 4 * 4;
  if (fw_out) *fw_out = fw;
  if (ow_out) *ow_out = ow;
  Carve c;
  c.take((size_t)s->d.L.n * fw * 8);
  c.take((size_t)s->d.L.n * fw * 8);
  c.take((size_t)std::max<uint64_t>(1, s->n_meas) * ow * 8);  // device record if output is host
  return c.off;
}

size_t qs_sim_sample_required_bytes(const qs_sim *s, uint64_t shots) {
  if (!s || shots == 0) return 0;
  return sample_bytes(s, shots, nullptr, nullptr);
}

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int qs_sim_sample(qs_sim *s, uint64_t shots, uint64_t seed, uint64_t *record, size_t record_words,
                  void *frame_ws, size_t frame_ws_bytes) {
  Range range_("qs_sim_sample");
  int rc = check_usable(s);
  if (rc) return rc;
  if (s->resumed)
    return fail(QS_ERR_STATE, "sampling replays the op log from |0...0>; a sim restored by "
                              "qs_sim_tableau_import has none (qs_sim_reset first)");
  if (shots == 0 || shots > kMaxShots) return fail(QS_ERR_ARG, "shots must be in [1, 2e9]");
  uint64_t fw, ow;
  const size_t need = sample_bytes(s, shots, &fw, &ow);
  const uint64_t M = s->n_meas;
  if (M && !record) return fail(QS_ERR_ARG, "record is NULL");
  if (record_words < M * ow) return fail(QS_ERR_SIZE, "record smaller than M * ceil(shots/64) words");
  if (frame_ws && frame_ws_bytes < need) return fail(QS_ERR_SIZE, "frame workspace too small");
  bool own = false;
  void *ws = frame_ws;
  if (!ws) {
    QS_CUDA(s, cudaMallocAsync(&ws, need, s->stream));
    own = true;
  }
  // frees the frames on every early return; the normal path frees them itself
  // and checks the result
  struct FramesGuard {
    qs_sim *s;
    void *ws;
    bool own;
    ~FramesGuard() {
      if (own && cudaFreeAsync(ws, s->stream) != cudaSuccess) cudaGetLastError();
    }
  } guard{s, ws, own};
  Carve c;
  uint8_t *b = static_cast<uint8_t *>(ws);
  const uint32_t n = s->d.L.n;
  uint64_t *FX = reinterpret_cast<uint64_t *>(b + c.take((size_t)n * fw * 8));
  uint64_t *FZ = reinterpret_cast<uint64_t *>(b + c.take((size_t)n * fw * 8));
  uint64_t *dout = reinterpret_cast<uint64_t *>(b + c.take((size_t)std::max<uint64_t>(1, M) * ow * 8));
  const bool out_dev = M ? is_device_ptr(record) : true;
  uint64_t *out = out_dev ? record : dout;
  if ((rc = upload_noise_targets(s))) return rc;
  tbegin(s->d.timer, QS_TIME_SAMPLE, s->stream);
  QS_CUDA(s, launch_frame_init(FX, FZ, n, (uint32_t)fw, seed, s->stream));
  s->launches += 1;
  std::vector<uint32_t> qtmp, seen(n, 0);
  uint32_t sid = 0;
  for (const Op &op : s->ops) {
    if (op.kind == Op::kHostLayer) {
      int slot;
      uint8_t *h = ring_slot(s, &slot);
      if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
      memcpy(h, op.packed.data(), op.packed.size() * 4);
      if ((rc = upload(s, slot, op.packed.size() * 4))) return rc;
      QS_CUDA(s, launch_frame_layer(FX, FZ, n, (uint32_t)fw, reinterpret_cast<uint32_t *>(s->dstage),
                                    (uint32_t)(op.packed.size() / 2), s->d.err, s->stream));
      s->launches += 1;
    } else if (op.kind == Op::kDevLayers) {
      if ((rc = run_dev_layers(s, FX, FZ, nullptr, (uint32_t)fw, op.dev, op.ptr.data(),
                               op.ptr.size() - 1, false)))
        return rc;
    } else if (op.kind == Op::kNoise) {
      if ((rc = replay_noise_dev(s, op, FX, FZ, (uint32_t)fw, (uint32_t)ow, seed))) return rc;
    } else {
      // measurement window: split into runs of distinct qubits (Sec. 5 processes
      // the measurements of one window in parallel)
      const uint32_t *qh;
      uint32_t cnt;
      if (op.kind == Op::kHostMeasure) {
        qh = op.qubits.data();
        cnt = (uint32_t)op.qubits.size();
      } else {
        qtmp.resize(op.count);
        QS_CUDA(s, cudaMemcpyAsync(qtmp.data(), op.dev, (size_t)op.count * 4, cudaMemcpyDeviceToHost,
                                   s->stream));
        QS_CUDA(s, cudaStreamSynchronize(s->stream));
        qh = qtmp.data();
        cnt = op.count;
      }
      const uint32_t chunk = (uint32_t)(s->plan.stage_bytes / 4);
      uint32_t start = 0;
      while (start < cnt) {
        if (++sid == 0) { std::fill(seen.begin(), seen.end(), 0); sid = 1; }
        uint32_t end = start;
        while (end < cnt && end - start < chunk && (qh[end] >= n || seen[qh[end]] != sid)) {
          if (qh[end] < n) seen[qh[end]] = sid;
          ++end;
        }
        int slot;
        uint8_t *h = ring_slot(s, &slot);
        if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
        memcpy(h, qh + start, (size_t)(end - start) * 4);
        if ((rc = upload(s, slot, (size_t)(end - start) * 4))) return rc;
        QS_CUDA(s, launch_frame_measure(FX, FZ, n, (uint32_t)fw,
                                        reinterpret_cast<uint32_t *>(s->dstage), end - start,
                                        op.m0 + start, s->d.record, out, shots, seed, s->d.err,
                                        s->stream));
        s->launches += (end - start + 65534) / 65535;
        start = end;
      }
    }
  }
  tend(s->d.timer, QS_TIME_SAMPLE, s->stream);
  if (!out_dev && M)
    QS_CUDA(s, cudaMemcpyAsync(record, dout, (size_t)(M * ow * 8), cudaMemcpyDeviceToHost, s->stream));
  guard.own = false;
  if (own) QS_CUDA(s, cudaFreeAsync(ws, s->stream));
  if (!out_dev) return qs_sim_sync(s);
  return QS_OK;
}

static size_t tableau_bytes(const Layout &L, int layout) {
  if (layout == QS_LAYOUT_NATIVE) return (2ull * L.n + 1) * L.cw * 8;
  return (2ull * L.n * 2 * L.k + (2ull * L.n + 63) / 64) * 8;
}

int qs_sim_tableau_export(qs_sim *s, int layout, void *dst, size_t dst_bytes, size_t *needed) {
  Range range_("qs_sim_tableau_export");
  int rc = check_usable(s);
  if (rc) return rc;
  if (layout != QS_LAYOUT_ROWS_PACKED && layout != QS_LAYOUT_NATIVE)
    return fail(QS_ERR_ARG, "unknown layout");
  const Layout &L = s->d.L;
  const uint32_t n = L.n, k = L.k;
  const size_t bytes = tableau_bytes(L, layout);
  if (needed) *needed = bytes;
  if (!dst) return QS_OK;
  if (dst_bytes < bytes) return fail(QS_ERR_SIZE, "export buffer too small");
  uint64_t *o = static_cast<uint64_t *>(dst);
  // cudaMemcpyDefault: dst may be host or device memory
  if (layout == QS_LAYOUT_NATIVE) {
    if ((rc = ensure_cols(s))) return rc;
    // columns of cw words out of the device's cs-word stride
    const size_t colw = (size_t)n * L.cw, dp = (size_t)L.cw * 8, sp = (size_t)L.cs * 8;
    QS_CUDA(s, cudaMemcpy2DAsync(o, dp, s->d.X, sp, dp, n, cudaMemcpyDefault, s->stream));
    QS_CUDA(s, cudaMemcpy2DAsync(o + colw, dp, s->d.Z, sp, dp, n, cudaMemcpyDefault, s->stream));
    QS_CUDA(s, cudaMemcpyAsync(o + 2 * colw, s->d.S, dp, cudaMemcpyDefault, s->stream));
    return qs_sim_sync(s);
  }
  if ((rc = ensure_rows(s))) return rc;
  const size_t dp = 2ull * k * 8, sp = (size_t)L.rs * 8, wb = (size_t)k * 8;
  QS_CUDA(s, cudaMemcpy2DAsync(o, dp, s->d.RX, sp, wb, n, cudaMemcpyDefault, s->stream));
  QS_CUDA(s, cudaMemcpy2DAsync(o + k, dp, s->d.RZ, sp, wb, n, cudaMemcpyDefault, s->stream));
  const size_t st = 64ull * k * L.rs;
  QS_CUDA(s, cudaMemcpy2DAsync(o + (size_t)n * 2 * k, dp, s->d.RX + st, sp, wb, n, cudaMemcpyDefault,
                               s->stream));
  QS_CUDA(s, cudaMemcpy2DAsync(o + (size_t)n * 2 * k + k, dp, s->d.RZ + st, sp, wb, n,
                               cudaMemcpyDefault, s->stream));
  std::vector<uint64_t> S(L.cs);
  QS_CUDA(s, cudaMemcpyAsync(S.data(), s->d.S, (size_t)L.cs * 8, cudaMemcpyDeviceToHost, s->stream));
  if ((rc = qs_sim_sync(s))) return rc;
  const size_t sw = (2ull * n + 63) / 64;
  std::vector<uint64_t> sig(sw, 0);
  for (uint64_t i = 0; i < 2ull * n; ++i) {
    const uint64_t pr = i < n ? i : 64ull * k + (i - n);
    if ((S[pr >> 6] >> (pr & 63)) & 1u) sig[i >> 6] |= 1ull << (i & 63);
  }
  QS_CUDA(s, cudaMemcpy(o + 2ull * n * 2 * k, sig.data(), sw * 8, cudaMemcpyDefault));
  return QS_OK;
}

// Words of a W-word NATIVE vector that hold bits belonging to no generator
// (packed numbers [n, 64 k) and [64 k + n, 64 W)), with those bits' mask.
static std::vector<std::pair<uint32_t, uint64_t>> native_padding(const Layout &L) {
  const uint64_t n = L.n, k = L.k;
  std::vector<std::pair<uint32_t, uint64_t>> pads;
  for (uint64_t w = 0; w < L.cw; ++w) {
    uint64_t pad = 0;
    for (int b = 0; b < 64; ++b) {
      const uint64_t g = 64 * w + b;
      if (!(g < n || (g >= 64 * k && g < 64 * k + n))) pad |= 1ull << b;
    }
    if (pad) pads.emplace_back((uint32_t)w, pad);
  }
  return pads;
}

int qs_sim_tableau_import(qs_sim *s, int layout, const void *src, size_t src_bytes,
                          const uint8_t *record, uint64_t record_count) {
  Range range_("qs_sim_tableau_import");
  int rc = check_usable(s);
  if (rc) return rc;
  if (s->d.inverse) return fail(QS_ERR_ARG, "qs_sim_tableau_import is not supported in inverse-tableau mode");
  if (layout != QS_LAYOUT_ROWS_PACKED && layout != QS_LAYOUT_NATIVE)
    return fail(QS_ERR_ARG, "unknown layout");
  const Layout &L = s->d.L;
  const uint32_t n = L.n, k = L.k;
  const size_t bytes = tableau_bytes(L, layout);
  if (!src || src_bytes < bytes) return fail(QS_ERR_SIZE, "import buffer smaller than the tableau");
  if (record_count > s->d.record_cap)
    return fail(QS_ERR_SIZE, "record capacity exceeded (qs_options.record_capacity)");
  if (record_count && !record) return fail(QS_ERR_ARG, "record is NULL");
  const uint64_t *in = static_cast<const uint64_t *>(src);
  if (layout == QS_LAYOUT_NATIVE) {
    const auto pads = native_padding(L);
    for (uint64_t c = 0; c < 2ull * n + 1; ++c)  // n X columns, n Z columns, the signs
      for (const auto &pw : pads)
        if (in[c * L.cw + pw.first] & pw.second)
          return fail(QS_ERR_ARG, "vector " + std::to_string(c) + " has bits outside the generators "
                                  "(word " + std::to_string(pw.first) + ")");
    const size_t colw = (size_t)n * L.cw, sp = (size_t)L.cw * 8, dp = (size_t)L.cs * 8;
    const size_t allw = (size_t)L.ncols * L.cs;  // padding qubit columns and words stay zero
    QS_CUDA(s, cudaMemsetAsync(s->d.X, 0, allw * 8, s->stream));
    QS_CUDA(s, cudaMemsetAsync(s->d.Z, 0, allw * 8, s->stream));
    QS_CUDA(s, cudaMemsetAsync(s->d.S, 0, dp, s->stream));
    QS_CUDA(s, cudaMemcpy2DAsync(s->d.X, dp, in, sp, sp, n, cudaMemcpyHostToDevice, s->stream));
    QS_CUDA(s, cudaMemcpy2DAsync(s->d.Z, dp, in + colw, sp, sp, n, cudaMemcpyHostToDevice, s->stream));
    QS_CUDA(s, cudaMemcpyAsync(s->d.S, in + 2 * colw, sp, cudaMemcpyHostToDevice, s->stream));
  } else {
    // bits of qubits >= n in the last word of each row must be zero
    if (n & 63) {
      const uint64_t pad = ~0ull << (n & 63);
      for (uint64_t i = 0; i < 2ull * n; ++i)
        if ((in[i * 2 * k + k - 1] | in[i * 2 * k + 2 * k - 1]) & pad)
          return fail(QS_ERR_ARG, "row " + std::to_string(i) + " has bits beyond qubit n - 1");
    }
    const uint64_t *sig = in + 2ull * n * 2 * k;
    std::vector<uint64_t> S(L.cs, 0);
    for (uint64_t i = 0; i < 2ull * n; ++i) {
      const uint64_t pr = i < n ? i : 64ull * k + (i - n);
      if ((sig[i >> 6] >> (i & 63)) & 1u) S[pr >> 6] |= 1ull << (pr & 63);
    }
    const size_t rowb = (size_t)L.nrows * L.rs * 8;
    QS_CUDA(s, cudaMemsetAsync(s->d.RX, 0, rowb, s->stream));
    QS_CUDA(s, cudaMemsetAsync(s->d.RZ, 0, rowb, s->stream));
    const size_t sp = 2ull * k * 8, dp = (size_t)L.rs * 8, wb = (size_t)k * 8;
    const size_t st = 64ull * k * L.rs;
    QS_CUDA(s, cudaMemcpy2DAsync(s->d.RX, dp, in, sp, wb, n, cudaMemcpyHostToDevice, s->stream));
    QS_CUDA(s, cudaMemcpy2DAsync(s->d.RZ, dp, in + k, sp, wb, n, cudaMemcpyHostToDevice, s->stream));
    QS_CUDA(s, cudaMemcpy2DAsync(s->d.RX + st, dp, in + (size_t)n * 2 * k, sp, wb, n,
                                 cudaMemcpyHostToDevice, s->stream));
    QS_CUDA(s, cudaMemcpy2DAsync(s->d.RZ + st, dp, in + (size_t)n * 2 * k + k, sp, wb, n,
                                 cudaMemcpyHostToDevice, s->stream));
    QS_CUDA(s, cudaMemcpyAsync(s->d.S, S.data(), (size_t)L.cs * 8, cudaMemcpyHostToDevice, s->stream));
    // the host vector must outlive the copy
    QS_CUDA(s, cudaStreamSynchronize(s->stream));
  }
  if (record_count) {
    QS_CUDA(s, cudaMemcpyAsync(s->d.record, record, record_count, cudaMemcpyHostToDevice, s->stream));
    QS_CUDA(s, cudaMemsetAsync(s->d.kinds, 2, record_count, s->stream));
  }
  QS_CUDA(s, cudaMemsetAsync(s->d.err, 0, 4, s->stream));
  QS_CUDA(s, launch_reset_meas_state(s->d, s->stream));
  s->launches += 1;
  QS_CUDA(s, cudaStreamSynchronize(s->stream));  // the host buffers may go once this returns
  s->rows_valid = layout == QS_LAYOUT_ROWS_PACKED;
  s->cols_valid = layout == QS_LAYOUT_NATIVE;
  s->n_meas = record_count;
  s->n_noise = 0;
  s->ops.clear();
  s->noise_dev_ops = 0;
  s->resumed = true;
  return QS_OK;
}

int qs_sim_qubit_signs(qs_sim *s, uint64_t *dst, size_t dst_words) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (!s->d.inverse) return fail(QS_ERR_STATE, "qubit signs exist in inverse-tableau mode only");
  if (!dst) return fail(QS_ERR_ARG, "dst is NULL");
  const size_t w = s->d.L.k;  // ceil(n / 64)
  if (dst_words < 2 * w) return fail(QS_ERR_SIZE, "dst smaller than 2 ceil(n/64) words");
  const cudaMemcpyKind kind = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  QS_CUDA(s, cudaMemcpyAsync(dst, s->d.qsig, w * 8, kind, s->stream));
  QS_CUDA(s, cudaMemcpyAsync(dst + w, s->d.qsig + s->d.L.rs, w * 8, kind, s->stream));
  return qs_sim_sync(s);
}

int qs_sim_export_rows(qs_sim *s, const uint32_t *rows, uint32_t count, uint64_t *dst) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (count && (!rows || !dst)) return fail(QS_ERR_ARG, "NULL argument");
  const Layout &L = s->d.L;
  const uint32_t n = L.n, k = L.k;
  for (uint32_t i = 0; i < count; ++i)
    if (rows[i] >= 2 * n) return fail(QS_ERR_ARG, "row index >= 2n");
  if (count == 0) return QS_OK;
  if ((rc = ensure_rows(s))) return rc;
  std::vector<uint64_t> S(L.cs);
  QS_CUDA(s, cudaMemcpyAsync(S.data(), s->d.S, (size_t)L.cs * 8, cudaMemcpyDeviceToHost, s->stream));
  const size_t per = 2ull * k + 1;
  for (uint32_t i = 0; i < count; ++i) {
    const uint64_t pr = rows[i] < n ? rows[i] : 64ull * k + (rows[i] - n);
    QS_CUDA(s, cudaMemcpyAsync(dst + i * per, s->d.RX + pr * L.rs, (size_t)k * 8,
                               cudaMemcpyDeviceToHost, s->stream));
    QS_CUDA(s, cudaMemcpyAsync(dst + i * per + k, s->d.RZ + pr * L.rs, (size_t)k * 8,
                               cudaMemcpyDeviceToHost, s->stream));
  }
  if ((rc = qs_sim_sync(s))) return rc;
  for (uint32_t i = 0; i < count; ++i) {
    const uint64_t pr = rows[i] < n ? rows[i] : 64ull * k + (rows[i] - n);
    dst[i * per + 2 * k] = (S[pr >> 6] >> (pr & 63)) & 1u;
  }
  return QS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free frame sampling (qs_sim_sample_noalloc in include/qs.h).
//
// Some callers cannot allocate device memory at the moment they want samples:
// a serving process that reserved the whole GPU for its own pool up front, a
// host framework whose caching allocator must own every byte, or a latency
// loop that cannot take the device-wide synchronisation of cudaFree. For them
// the Pauli frames live in one file-scope device array of fixed size instead
// of a caller workspace or cudaMallocAsync. Every GPU that loads this library
// holds the array until the process exits; all calls share it.
// ---------------------------------------------------------------------------
#include <mutex>

static __device__ __align__(256) uint64_t g_noalloc_frames[QS_NOALLOC_SCRATCH_BYTES / 8];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices] = {};
// host bitmap used to cut measurement windows into runs of distinct qubits
uint64_t g_noalloc_seen[(kMaxQubits + 63) / 64];
}  // namespace

// Set-up, once per device with that device current: the host-side name of the
// array is not a device address, so ask the runtime for it (this also loads
// the array onto the device). Callers hold g_noalloc_mu or are qs_sim_create.
static cudaError_t noalloc_setup_locked(void **addr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_frames);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_noalloc_addr[dev] = p;
  }
  *addr = g_noalloc_addr[dev];
  return cudaSuccess;
}

static cudaError_t noalloc_setup(void **addr) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  return noalloc_setup_locked(addr);
}

extern "C" int qs_sim_sample_noalloc(qs_sim *s, uint64_t shots, uint64_t seed, uint64_t *record,
                                     size_t record_words) {
  Range range_("qs_sim_sample_noalloc");
  int rc = check_usable(s);
  if (rc) return rc;
  if (s->resumed)
    return fail(QS_ERR_STATE, "sampling replays the op log from |0...0>; a sim restored by "
                              "qs_sim_tableau_import has none (qs_sim_reset first)");
  if (shots == 0 || shots > kMaxShots) return fail(QS_ERR_ARG, "shots must be in [1, 2e9]");
  const uint32_t n = s->d.L.n;
  const uint64_t M = s->n_meas;
  const uint64_t ow = (shots + 63) / 64, fw = (ow + 3) / 4 * 4;
  const size_t fbytes = (((size_t)n * fw * 8) + 255) & ~size_t(255);
  const size_t need = 2 * fbytes + (size_t)std::max<uint64_t>(1, M) * ow * 8;
  if (fw > 0xFFFFFFFFull || need > (size_t)QS_NOALLOC_SCRATCH_BYTES) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "qs_sim_sample_noalloc needs %zu bytes of frames for n = %u and %llu shots; the "
             "static scratch holds %u bytes",
             need, n, (unsigned long long)shots, (unsigned)QS_NOALLOC_SCRATCH_BYTES);
    return fail(QS_ERR_SIZE, buf);
  }
  if (M && !record) return fail(QS_ERR_ARG, "record is NULL");
  if (record_words < M * ow) return fail(QS_ERR_SIZE, "record smaller than M * ceil(shots/64) words");
  int dev = 0;
  QS_CUDA(s, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(QS_ERR_ARG, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  void *addr = nullptr;
  {
    // normally done at qs_sim_create; a failure here leaves the sim usable
    cudaError_t e = noalloc_setup_locked(&addr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(QS_ERR_CUDA, std::string("the static sampling array could not be placed on the "
                                           "device: ") + cudaGetErrorString(e));
    }
  }
  uint8_t *base = static_cast<uint8_t *>(addr);
  uint64_t *FX = reinterpret_cast<uint64_t *>(base);
  uint64_t *FZ = reinterpret_cast<uint64_t *>(base + fbytes);
  uint64_t *dout = reinterpret_cast<uint64_t *>(base + 2 * fbytes);
  const bool out_dev = M ? is_device_ptr(record) : true;
  uint64_t *out = out_dev ? record : dout;
  // X~ is cleared to zero and Z~ fully rewritten by the init launch
  QS_CUDA(s, launch_frame_init(FX, FZ, n, (uint32_t)fw, seed, s->stream));
  s->launches += 1;
  for (const Op &op : s->ops) {
    if (op.kind == Op::kHostLayer) {
      int slot;
      uint8_t *h = ring_slot(s, &slot);
      if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
      memcpy(h, op.packed.data(), op.packed.size() * 4);
      if ((rc = upload(s, slot, op.packed.size() * 4))) return rc;
      QS_CUDA(s, launch_frame_layer(FX, FZ, n, (uint32_t)fw, reinterpret_cast<uint32_t *>(s->dstage),
                                    (uint32_t)(op.packed.size() / 2), s->d.err, s->stream));
      s->launches += 1;
    } else if (op.kind == Op::kDevLayers) {
      for (size_t l = 0; l + 1 < op.ptr.size(); ++l) {
        const int64_t a = op.ptr[l], cnt = op.ptr[l + 1] - a;
        QS_CUDA(s, launch_frame_layer(FX, FZ, n, (uint32_t)fw, op.dev + 2 * a, (uint32_t)cnt,
                                      s->d.err, s->stream));
        if (cnt) s->launches += 1;
      }
    } else if (op.kind == Op::kNoise) {
      if ((rc = replay_noise(s, op, FX, FZ, (uint32_t)fw, (uint32_t)ow, seed))) return rc;
    } else if (op.kind == Op::kDevMeasure) {
      // the list stays on the device: one launch per measurement keeps repeated
      // qubits in program order without reading the list back
      for (uint32_t i = 0; i < op.count; ++i) {
        QS_CUDA(s, launch_frame_measure(FX, FZ, n, (uint32_t)fw, op.dev + i, 1, op.m0 + i,
                                        s->d.record, out, shots, seed, s->d.err, s->stream));
        s->launches += 1;
      }
    } else {
      const uint32_t *qh = op.qubits.data();
      const uint32_t cnt = (uint32_t)op.qubits.size();
      const uint32_t chunk = (uint32_t)(s->plan.stage_bytes / 4);
      uint32_t start = 0;
      while (start < cnt) {
        uint32_t end = start;
        while (end < cnt && end - start < chunk &&
               !((g_noalloc_seen[qh[end] >> 6] >> (qh[end] & 63)) & 1u)) {
          g_noalloc_seen[qh[end] >> 6] |= 1ull << (qh[end] & 63);
          ++end;
        }
        for (uint32_t i = start; i < end; ++i) g_noalloc_seen[qh[i] >> 6] = 0;
        int slot;
        uint8_t *h = ring_slot(s, &slot);
        if (!h) return cuda_fail(s, cudaGetLastError(), "staging event");
        memcpy(h, qh + start, (size_t)(end - start) * 4);
        if ((rc = upload(s, slot, (size_t)(end - start) * 4))) return rc;
        QS_CUDA(s, launch_frame_measure(FX, FZ, n, (uint32_t)fw,
                                        reinterpret_cast<uint32_t *>(s->dstage), end - start,
                                        op.m0 + start, s->d.record, out, shots, seed, s->d.err,
                                        s->stream));
        s->launches += (end - start + 65534) / 65535;
        start = end;
      }
    }
  }
  if (!out_dev && M)
    QS_CUDA(s, cudaMemcpyAsync(record, dout, (size_t)(M * ow * 8), cudaMemcpyDeviceToHost, s->stream));
  if (!out_dev) return qs_sim_sync(s);
  return QS_OK;
}
