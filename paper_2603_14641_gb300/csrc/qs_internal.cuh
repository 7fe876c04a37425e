// Internal declarations shared by the kernels and the C-ABI runtime of libqs.
//
// Memory layout in HBM (one sim of n qubits, k = ceil(n/64)):
//   Column-major tableau (gate layers, Sec. 4.3 "Memory Layout"):
//     X[q][w], Z[q][w] for q < ncols (= n rounded up to 256), w < cs
//     (cs = 2k rounded up to 4 words; both rounded further up to 2 KB strides
//     where that costs at most 1 %, see pad_stride). Bit b of word w is packed
//     row 64 w + b.
//     Packed rows: destabilizer D_i is row i, stabilizer S_i is row 64 k + i;
//     the remaining packed rows are zero padding and stay zero under every gate.
//   Signs S[w], w < cs: bit b of word w = sign bit of packed row 64 w + b
//     (forward, per-generator signs; untouched by the transposes).
//   Row-major tableau (measurement, Sec. 4.3): RX[r][u], RZ[r][u] for packed
//     row r < 64 cs and u < rs (= ncols / 64); bit j of word u = qubit 64 u + j.
// All words are 64-bit; column and row starts are 32-byte aligned so that
// 128-bit vector accesses are aligned.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include <string>
#include <vector>

#include "../../include/qs.h"

namespace qs {

constexpr int kDetBlocks = 152;     // chunks of the deterministic product (one per SM)
constexpr int kMeasStateWords = 16; // per-measurement device state
constexpr int kInvChunks = 512;     // row chunks of the inverse-mode target pass

// device error flags (sticky, cleared by reset)
enum : uint32_t {
  kErrOddPhase = 1u,    // a rowsum produced an odd power of i
  kErrDetProduct = 2u,  // deterministic product was not +-Z_q
  kErrBadGate = 4u,     // packed gate with out-of-range qubit or type
  kErrBadQubit = 8u,    // measured qubit out of range
  kErrTimeout = 16u,    // a bounded device wait ran out
};

// measurement state words (device), indices into MeasState array
enum : int {
  kMsPivot = 0,      // packed pivot row (int64), or INT64_MAX if none
  kMsDetCross = 1,   // XOR of cross parities from the combine pass
  kMsDetXZ = 2,      // sum of popc(Xtot & Ztot) (must be 0)
};

struct Layout {
  uint32_t n, k, cs, ncols, rs;
  uint64_t nrows;  // 64 * cs
  uint32_t cw;     // 2k rounded up to 4: the column width of QS_LAYOUT_NATIVE (cs >= cw)
};

// A stride of w words is rounded up to a multiple of 256 words (2 KB) when
// that adds at most 1 %: the TMA transposes between the two layouts measured
// 5.8 TB/s in both directions at 180,000 qubits with both strides multiples
// of 2 KB (column stride 5,632 words) against 4.4-5.6 TB/s with 5,628.
inline uint32_t pad_stride(uint32_t w) {
  const uint32_t r = (w + 255) / 256 * 256;
  return (uint64_t)(r - w) * 100 <= w ? r : w;
}

inline Layout make_layout(uint32_t n) {
  Layout L;
  L.n = n;
  L.k = (n + 63) / 64;
  L.cw = ((2 * L.k) + 3) / 4 * 4;
  L.cs = pad_stride(L.cw);
  L.ncols = pad_stride((n + 255) / 256 * 4) * 64;
  L.rs = L.ncols / 64;
  L.nrows = 64ull * L.cs;
  return L;
}

// ------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): device implementation.
// ------------------------------------------------------------------------
struct P4 { uint64_t v[4]; };

__device__ __forceinline__ P4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                             uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    uint64_t hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
    uint64_t hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
  P4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

constexpr uint64_t kCoinKey = 0x51A7Eull;
constexpr uint64_t kFrameKey = 0xF4A3Eull;
constexpr uint64_t kNoiseKey = 0xE5505ull;

// Runs `set` (kernel attribute calls) once per device ordinal, safely from
// several host threads: `done` holds one bit per device already set (ordinals
// >= 64 set every time). Setting an attribute twice is harmless.
template <class F>
inline cudaError_t once_per_device(std::atomic<uint64_t> &done, F set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return set();
  const uint64_t bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Optional CUDA-event timing of kernel classes (qs_sim_set_timing): begin/end
// record an event pair on the stream around a group of launches; pairs are
// resolved into elapsed milliseconds once their end event has completed.
// Kinds are the QS_TIME_* values of qs.h.
struct KernelTimer {
  double ms[QS_NUM_TIME_KINDS] = {};
  uint64_t count[QS_NUM_TIME_KINDS] = {};
  struct Pair { int kind; cudaEvent_t a, b; };
  std::vector<Pair> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open[QS_NUM_TIME_KINDS] = {};

  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
  }
  void begin(int kind, cudaStream_t s) {
    if (open[kind]) { pool.push_back(open[kind]); open[kind] = nullptr; }  // left open by an error
    cudaEvent_t e = get();
    if (e && cudaEventRecord(e, s) == cudaSuccess) open[kind] = e;
  }
  void end(int kind, cudaStream_t s) {
    cudaEvent_t a = open[kind];
    open[kind] = nullptr;
    if (!a) return;
    cudaEvent_t b = get();
    if (!b || cudaEventRecord(b, s) != cudaSuccess) { pool.push_back(a); return; }
    pending.push_back({kind, a, b});
  }
  // adds the pairs whose end event has completed (all of them after a sync)
  void resolve() {
    size_t keep = 0;
    for (size_t i = 0; i < pending.size(); ++i) {
      Pair p = pending[i];
      if (cudaEventQuery(p.b) != cudaSuccess) { cudaGetLastError(); pending[keep++] = p; continue; }
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        ms[p.kind] += t;
        count[p.kind] += 1;
      } else {
        cudaGetLastError();
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.resize(keep);
  }
  void clear() {
    resolve();
    for (int k = 0; k < QS_NUM_TIME_KINDS; ++k) { ms[k] = 0; count[k] = 0; }
  }
  ~KernelTimer() {
    for (auto &p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
    for (auto e : open) if (e) cudaEventDestroy(e);
  }
};

// begin/end on an optional timer
inline void tbegin(KernelTimer *t, int kind, cudaStream_t s) { if (t) t->begin(kind, s); }
inline void tend(KernelTimer *t, int kind, cudaStream_t s) { if (t) t->end(kind, s); }

// ------------------------------------------------------------------------
// Launchers (each returns cudaGetLastError() after the launch).
// ------------------------------------------------------------------------
struct Dev {
  Layout L;
  uint64_t *X, *Z, *S;     // column-major tableau + signs
  uint64_t *RX, *RZ;       // row-major tableau
  uint32_t *colx;          // gathered x column, 2 * cs uint32 (= cs words)
  int64_t *mst;            // measurement state (kMeasStateWords)
  uint64_t *det_x, *det_z; // kDetBlocks * rs words each
  int32_t *det_scal;       // kDetBlocks partial phase sums
  uint32_t *err;           // sticky error flags
  uint8_t *record;         // record bytes
  uint8_t *kinds;          // per record entry: 1 probabilistic, 0 deterministic, 2 restored
  uint64_t record_cap;
  int sms;                 // multiprocessor count of the device
  bool wide_offsets;       // 64-bit row offsets in the blocked apply pass at any size
  bool step_symbolic;      // blocked symbolic pass as one launch per step at any size
  KernelTimer *timer;      // CUDA-event timing of kernel classes, or nullptr (off)
  bool inverse;            // inverse-tableau mode (qubit-indexed signs, Alg. 1 measurement)
  uint64_t *qsig;          // inverse mode: S_S then S_D, rs words each
  uint64_t *inv_part;      // inverse mode: measurement partials, 6 * kInvChunks * rs words
};

cudaError_t launch_init(const Dev &d, const uint8_t *initstate_dev, cudaStream_t s);
cudaError_t launch_gate_layer(const Dev &d, const uint32_t *packed, uint32_t n_gates,
                              cudaStream_t s);
// frames: column-major frame matrices FX/FZ [n][fw] words (fw multiple of 2)
cudaError_t launch_frame_layer(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw,
                               const uint32_t *packed, uint32_t n_gates, uint32_t *err,
                               cudaStream_t s);
cudaError_t launch_to_rows(const Dev &d, cudaStream_t s);
cudaError_t launch_to_cols(const Dev &d, cudaStream_t s);
// one Z-measurement of qubits[i] with record index midx
cudaError_t launch_measure_one(const Dev &d, const uint32_t *qubits, uint32_t i, uint64_t midx,
                               qs_key key, cudaStream_t s, int *launches);
cudaError_t launch_frame_init(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw, uint64_t seed,
                              cudaStream_t s);
cudaError_t launch_frame_measure(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw,
                                 const uint32_t *qubits, uint32_t count, uint64_t m0,
                                 const uint8_t *ref, uint64_t *out, uint64_t shots, uint64_t seed,
                                 uint32_t *err, cudaStream_t s);
// noise op e (QS_NOISE_* kind) on targets[0..count) (pairs for DEPOLARIZE2,
// count = number of pairs), global target index i0 + local index; shot words
// 0..ow-1; a shot fires iff its 32-bit draw u < thr (thr = 2^32: always)
cudaError_t launch_frame_noise(uint64_t *FX, uint64_t *FZ, uint32_t fw, uint32_t ow,
                               const uint32_t *targets, uint32_t count, uint32_t i0, int kind,
                               uint64_t thr, uint64_t e, uint64_t seed, cudaStream_t s);
cudaError_t launch_reset_meas_state(const Dev &d, cudaStream_t s);
// column q = qubits[i] of the row-major x part into colx, pivot by atomicMin into mst
cudaError_t launch_gather(const Dev &d, const uint32_t *qubits, uint32_t i, cudaStream_t s);
// inverse-tableau mode (qs_inverse.cu)
cudaError_t launch_inv_init_signs(const Dev &d, const uint8_t *initstate_dev, cudaStream_t s);
cudaError_t launch_inv_gate_layer(const Dev &d, const uint32_t *packed, uint32_t n_gates, cudaStream_t s);
size_t inv_scratch_words(const Layout &L);
cudaError_t launch_inv_measure_one(const Dev &d, const uint32_t *qubits, uint32_t i, uint64_t midx,
                                   qs_key key, cudaStream_t s, int *launches);
// a window of measurements qubits[0..count) with record indices m0.., two
// launches per measurement (plus two per window)
bool measure_window_supported(const Layout &L);
cudaError_t launch_measure_window(const Dev &d, const uint32_t *qubits, uint32_t count,
                                  uint64_t m0, qs_key key, cudaStream_t s, int *launches);
// blocked measurement (scratch of blocked_scratch_bytes): one block measures up
// to 64 qubits of a window of count (record indices from m0), starting at the
// window position the scratch's cursor holds, and moves the cursor past the
// steps it measured (it stops before a deterministic outcome); blocks can be
// enqueued back to back. block_cursor gives the cursor's device address,
// set_block_cursor sets it on the stream.
size_t blocked_scratch_bytes(const Layout &L);
cudaError_t launch_measure_block(const Dev &d, void *scratch, const uint32_t *window, uint32_t count,
                                 uint64_t m0, qs_key key, cudaStream_t s, int *launches);
cudaError_t set_block_cursor(const Layout &L, void *scratch, uint32_t v, cudaStream_t s);
const uint32_t *block_cursor(const Layout &L, void *scratch);
// fused segment of L layers on a word-sliced, shared-memory-resident tableau
// (S == nullptr: frames, no signs); lptr: L + 1 device gate offsets
bool fused_fits(uint32_t n);
// max_gates: the largest layer of the segment (gates)
cudaError_t launch_fused_segment(uint64_t *X, uint64_t *Z, uint64_t *S, uint32_t n, uint32_t stride,
                                 uint32_t nwords, const uint32_t *packed, const int64_t *lptr,
                                 uint32_t L, uint32_t max_gates, uint32_t *err, cudaStream_t s);

}  // namespace qs
