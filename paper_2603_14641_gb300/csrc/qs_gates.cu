// Tableau initialisation and Clifford gate layers on the column-major tableau.
//
// Sec. 4.4 (Alg. 3) applies a window of gates on disjoint qubits to every
// generator row, words of a column in parallel; the update rules are those of
// Sec. 2.4 Eq. 4 (H, P, CX) and, for the rest of the 11-gate set of Sec. 6,
// their compositions (S^dag = S^3, CZ = H_t CX H_t, CY = S_t CX S_t^dag,
// SWAP, ISWAP = CZ, SWAP, S_a, S_b), evaluated in registers so that each gate
// still reads and writes every touched column word once.
//
// GB300 mapping: a thread owns one 128-bit pair of column words (128 rows)
// for a run of gates; its sign contributions stay in registers and leave the
// block as one 64-bit XOR atomic per word per gate group (the paper's
// CollapseSigns tree of Alg. 3 becomes a register XOR). The same kernel, with
// signs compiled out, evolves the Pauli frames of Sec. 5 (Alg. 9 reuses the
// gate kernel on frames).
#include <algorithm>

#include "qs_internal.cuh"
#include "qs_rules.cuh"

namespace qs {

__device__ __forceinline__ ulonglong2 ld2(const uint64_t *p) {
  return *reinterpret_cast<const ulonglong2 *>(p);
}
__device__ __forceinline__ void st2(uint64_t *p, ulonglong2 v) {
  *reinterpret_cast<ulonglong2 *>(p) = v;
}

__device__ __forceinline__ bool is_two_qubit(uint32_t t) { return t >= QS_CX && t <= QS_ISWAP; }

// ---------------------------------------------------------------------
// init: D_i = X_i, S_i = Z_i, signs of both rows of qubit i = initstate[i]
// (Sec. 4.1 Alg. 2 InitializeTableau; pattern of Sec. 2.5 Eq. 8).
// X and Z are zeroed beforehand by cudaMemsetAsync.
// ---------------------------------------------------------------------
__global__ void init_diag_kernel(uint64_t *__restrict__ X, uint64_t *__restrict__ Z, uint32_t n,
                                 uint32_t k, uint32_t cs) {
  uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint64_t bit = 1ull << (q & 63);
  X[(size_t)q * cs + (q >> 6)] = bit;        // destabilizer row q
  Z[(size_t)q * cs + k + (q >> 6)] = bit;    // stabilizer row 64 k + q
}

__global__ void init_signs_kernel(uint64_t *__restrict__ S, const uint8_t *__restrict__ init,
                                  uint32_t n, uint32_t k, uint32_t cs) {
  uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= cs) return;
  uint64_t v = 0;
  if (init != nullptr && w < 2 * k) {
    uint32_t base = (w < k ? w : w - k) * 64;
    for (uint32_t b = 0; b < 64; ++b) {
      uint32_t i = base + b;
      if (i < n && init[i]) v |= 1ull << b;
    }
  }
  S[w] = v;
}

cudaError_t launch_init(const Dev &d, const uint8_t *initstate_dev, cudaStream_t s) {
  const Layout &L = d.L;
  size_t colbytes = (size_t)L.ncols * L.cs * sizeof(uint64_t);
  cudaError_t e;
  if ((e = cudaMemsetAsync(d.X, 0, colbytes, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.Z, 0, colbytes, s)) != cudaSuccess) return e;
  init_diag_kernel<<<(L.n + 255) / 256, 256, 0, s>>>(d.X, d.Z, L.n, L.k, L.cs);
  init_signs_kernel<<<(L.cs + 255) / 256, 256, 0, s>>>(d.S, initstate_dev, L.n, L.k, L.cs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------
// gate layer
//   packed[2 g] = type << 24 | q0, packed[2 g + 1] = q1
//   block: P pair-threads x `lanes` gate lanes (P * lanes <= 256);
//   grid.x: gate groups of `lanes * gpl` gates; grid.y: chunks of P pairs.
// On the tableau a thread walks its gates two at a time: both gates' column
// words are loaded before either is stored (the gates of a layer touch
// disjoint columns), which doubles the bytes each thread keeps in flight -- at
// one gate per thread the kernel is bound by memory latency x bytes in flight
// (0.87 of the HBM peak at 180k qubits; 0.97 with two). Frames with short
// columns (many gate lanes per block) keep one gate per thread.
// ---------------------------------------------------------------------
struct GateIn {
  uint32_t type, qa, qb;
  ulonglong2 x1, z1, x2, z2;
};

// Reads the record of gate g and the column words it needs; false for an
// invalid record (flagged, skipped).
template <bool SIGNS>
__device__ __forceinline__ bool gate_load(GateIn &in, uint32_t g, const uint32_t *__restrict__ packed,
                                          uint64_t *X, uint64_t *Z, uint32_t n, uint32_t cs,
                                          size_t off, bool flag, uint32_t *err) {
  const uint32_t w0 = __ldg(packed + 2 * g), qb = __ldg(packed + 2 * g + 1);
  const uint32_t type = w0 >> 24, qa = w0 & 0xFFFFFFu;
  const bool two = is_two_qubit(type);
  if (qa >= n || type >= QS_NUM_GATE_TYPES || (two && (qb >= n || qb == qa))) {
    if (flag) atomicOr(err, kErrBadGate);
    return false;
  }
  in.type = type;
  in.qa = qa;
  in.qb = qb;
  const uint64_t *xa = X + (size_t)qa * cs + off, *za = Z + (size_t)qa * cs + off;
  const uint64_t *xb = X + (size_t)qb * cs + off, *zb = Z + (size_t)qb * cs + off;
  const ulonglong2 zero = make_ulonglong2(0, 0);
  in.x1 = in.z1 = in.x2 = in.z2 = zero;
  switch (type) {
    case QS_X: if (SIGNS) in.z1 = ld2(za); break;
    case QS_Z: if (SIGNS) in.x1 = ld2(xa); break;
    case QS_Y: if (SIGNS) { in.x1 = ld2(xa); in.z1 = ld2(za); } break;
    case QS_H: case QS_S: case QS_SDG: in.x1 = ld2(xa); in.z1 = ld2(za); break;
    case QS_CX: case QS_CZ: case QS_CY: case QS_SWAP: case QS_ISWAP:
      in.x1 = ld2(xa); in.z1 = ld2(za); in.x2 = ld2(xb); in.z2 = ld2(zb); break;
    default: break;  // QS_I
  }
  return true;
}

// Applies the rules of qs_rules.cuh to both words and stores the columns the
// gate changes.
template <bool SIGNS>
__device__ __forceinline__ void gate_apply(GateIn &in, ulonglong2 &sacc, uint64_t *X, uint64_t *Z,
                                           uint32_t cs, size_t off) {
  uint64_t *xa = X + (size_t)in.qa * cs + off, *za = Z + (size_t)in.qa * cs + off;
  uint64_t *xb = X + (size_t)in.qb * cs + off, *zb = Z + (size_t)in.qb * cs + off;
  uint64_t s0 = 0, s1 = 0;
  uint64_t a0 = in.x1.x, b0 = in.z1.x, c0 = in.x2.x, d0 = in.z2.x;
  uint64_t a1 = in.x1.y, b1 = in.z1.y, c1 = in.x2.y, d1 = in.z2.y;
  rule<SIGNS>(in.type, a0, b0, c0, d0, s0);
  rule<SIGNS>(in.type, a1, b1, c1, d1, s1);
  in.x1 = make_ulonglong2(a0, a1);
  in.z1 = make_ulonglong2(b0, b1);
  in.x2 = make_ulonglong2(c0, c1);
  in.z2 = make_ulonglong2(d0, d1);
  if (SIGNS) { sacc.x ^= s0; sacc.y ^= s1; }
  switch (in.type) {
    case QS_H: st2(xa, in.x1); st2(za, in.z1); break;
    case QS_S: case QS_SDG: st2(za, in.z1); break;
    case QS_CX: st2(xb, in.x2); st2(za, in.z1); break;
    case QS_CZ: st2(za, in.z1); st2(zb, in.z2); break;
    case QS_CY: st2(za, in.z1); st2(xb, in.x2); st2(zb, in.z2); break;
    case QS_SWAP: case QS_ISWAP:
      st2(xa, in.x1); st2(za, in.z1); st2(xb, in.x2); st2(zb, in.z2); break;
    default: break;  // I, X, Y, Z change signs only
  }
}

template <bool SIGNS, int INFLIGHT>
__global__ void __launch_bounds__(256, INFLIGHT == 2 ? 4 : 6)
gate_layer_kernel(uint64_t *__restrict__ X, uint64_t *__restrict__ Z, uint64_t *__restrict__ S,
                  uint32_t n, uint32_t cs, const uint32_t *__restrict__ packed, uint32_t n_gates,
                  uint32_t P, uint32_t lanes, uint32_t gpl, uint32_t *__restrict__ err) {
  const uint32_t npairs = cs >> 1;
  const uint32_t t = threadIdx.x;
  const uint32_t lane = t / P;
  const uint32_t pair = blockIdx.y * P + (t - lane * P);
  const bool active = pair < npairs;
  const uint32_t group = lanes * gpl;
  const uint32_t g0 = blockIdx.x * group;
  const uint32_t g1 = min(g0 + group, n_gates);
  ulonglong2 sacc = make_ulonglong2(0, 0);

  if (active) {
    const size_t off = 2 * (size_t)pair;
    const bool flag = pair == 0;
    for (uint32_t g = g0 + lane; g < g1; g += INFLIGHT * lanes) {
      GateIn in[INFLIGHT];
      bool ok[INFLIGHT];
#pragma unroll
      for (int u = 0; u < INFLIGHT; ++u)
        ok[u] = g + u * lanes < g1 &&
                gate_load<SIGNS>(in[u], g + u * lanes, packed, X, Z, n, cs, off, flag, err);
#pragma unroll
      for (int u = 0; u < INFLIGHT; ++u)
        if (ok[u]) gate_apply<SIGNS>(in[u], sacc, X, Z, cs, off);
    }
  }
  if (SIGNS) {
    if (lanes > 1) {
      __shared__ ulonglong2 red[256];
      red[t] = sacc;
      __syncthreads();
      if (t < P) {
        for (uint32_t l = 1; l < lanes; ++l) {
          ulonglong2 v = red[l * P + t];
          sacc.x ^= v.x; sacc.y ^= v.y;
        }
      }
    }
    if (active && lane == 0) {
      if (sacc.x) atomicXor(reinterpret_cast<unsigned long long *>(S + 2 * (size_t)pair), sacc.x);
      if (sacc.y) atomicXor(reinterpret_cast<unsigned long long *>(S + 2 * (size_t)pair + 1), sacc.y);
    }
  }
}

struct GateGrid {
  dim3 grid, block;
  uint32_t P, lanes, gpl;
};

// Launch shape: P pair-threads per gate lane (a column chunk of up to 256
// pairs = 32 KB), as many gate lanes as fit 256 threads, and enough gates per
// lane that the grid covers the 152 SMs several times over while each block
// still amortises its sign atomics over several gates.
static GateGrid gate_grid(uint32_t npairs, uint32_t n_gates) {
  GateGrid g;
  g.P = std::min<uint32_t>(npairs, 256);
  g.lanes = std::max<uint32_t>(1, 256 / g.P);
  uint32_t chunks = (npairs + g.P - 1) / g.P;
  uint64_t slots = (n_gates + g.lanes - 1) / g.lanes;
  uint64_t want_blocks = 8ull * 152;
  uint64_t gpl = (slots * chunks + want_blocks - 1) / want_blocks;
  g.gpl = (uint32_t)std::min<uint64_t>(64, std::max<uint64_t>(4, gpl));
  uint64_t group = (uint64_t)g.lanes * g.gpl;
  g.grid = dim3((uint32_t)((n_gates + group - 1) / group), chunks, 1);
  g.block = dim3(g.P * g.lanes, 1, 1);
  return g;
}

cudaError_t launch_gate_layer(const Dev &d, const uint32_t *packed, uint32_t n_gates,
                              cudaStream_t s) {
  if (n_gates == 0) return cudaSuccess;
  GateGrid g = gate_grid(d.L.cs / 2, n_gates);
  gate_layer_kernel<true, 2><<<g.grid, g.block, 0, s>>>(d.X, d.Z, d.S, d.L.n, d.L.cs, packed, n_gates,
                                                     g.P, g.lanes, g.gpl, d.err);
  return cudaGetLastError();
}

cudaError_t launch_frame_layer(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw,
                               const uint32_t *packed, uint32_t n_gates, uint32_t *err,
                               cudaStream_t s) {
  if (n_gates == 0) return cudaSuccess;
  GateGrid g = gate_grid(fw / 2, n_gates);
  if (g.lanes == 1)  // long frame columns (>= 512 shot words): as the tableau, two gates in flight
    gate_layer_kernel<false, 2><<<g.grid, g.block, 0, s>>>(FX, FZ, nullptr, n, fw, packed, n_gates,
                                                        g.P, g.lanes, g.gpl, err);
  else
    gate_layer_kernel<false, 1><<<g.grid, g.block, 0, s>>>(FX, FZ, nullptr, n, fw, packed, n_gates,
                                                        g.P, g.lanes, g.gpl, err);
  return cudaGetLastError();
}

}  // namespace qs
