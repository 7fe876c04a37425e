// Blocked CHP measurement: up to 64 consecutive Z-measurements per pass over
// the row-major tableau, with exactly the result of measuring them one by one.
//
// Sequential CHP (Sec. 2.5) only ever (a) left-multiplies target rows by the
// current pivot row, (b) copies the pivot row into its destabilizer partner and
// (c) replaces the pivot row by (-1)^b Z_q. Which rows are pivots and targets
// depends only on the x bits of the measured columns, so the block is run in
// three parts:
//  1. symbolic pass: every packed row r carries C_r = its x bits at the block's
//     qubits q_0..q_{B-1} (one 64-bit word). Step j picks the pivot (smallest
//     stabilizer with bit j set), XORs the pivot's C into the targets and records
//     in M_r which steps targeted r; the destabilizer partner gets the pivot's C
//     (base = step j, M reset), the pivot row is marked. A step without a pivot
//     (deterministic outcome) ends the block there; it is measured afterwards by
//     the single-measurement path.
//  2. pivot rows: V_j = (V_{j'} ... over the steps j' that targeted row p_j, in
//     order) * original row p_j, built word-parallel; their signs follow from
//     the phase of a product of Paulis,
//       i^(2 sum r + sum |x_a & z_a| + 2 sum_{a<b} z_a . x_b - |X & Z|),
//     whose cross term is GF(2)-bilinear, so per-word popcounts summed over the
//     row (|x & z| of each V, of each original pivot row, parities
//     G[s][t] = z_{V_s} . x_{V_t}) are enough; the signs are then resolved in
//     step order by one thread.
//  3. one streaming pass: row r becomes (prod over s in M_r of V_s) * base_r,
//     base_r = its original value or V_j if it was replaced at step j; the XOR
//     accumulation reads the V words of a column chunk from shared memory, the
//     phase uses the same product formula with cross term
//     z_acc . x_base + sum_{s>t in M_r} G[s][t]. Pivot rows become +-Z_q.
// Per block the tableau is read and written once instead of once per
// measurement (the paper measures one qubit at a time, Alg. 2).
#include <algorithm>
#include <climits>

#include "qs_internal.cuh"

namespace qs {

constexpr int64_t kBlkNone = LLONG_MAX;
constexpr int32_t kBaseOrig = -1;
constexpr int32_t kBasePivot = 1000;  // base = kBasePivot + j: pivot row of step j
constexpr int kCW = 64;               // column words per phase-3 chunk

struct BlkState {
  int64_t slot[3];     // pivot search results, rotating
  int32_t len;         // steps completed in this block
  int32_t pad;
  int64_t piv[64];     // pivot row of each step
  uint64_t mpiv[64];   // steps that targeted the pivot row before it became pivot
  int32_t A[64];       // |x_V & z_V| mod 4 (summed over words)
  int32_t B0[64];      // |x & z| of the original pivot row
  int32_t Cp[64];      // parity of (z_V ^ z_orig) . x_orig
  int32_t rV[64];      // sign bit of V_j
  uint64_t G[64];      // G[s] bit t = parity(z_{V_s} . x_{V_t})
  uint32_t err;
};

__device__ __forceinline__ int m4(int v) { return ((v % 4) + 4) % 4; }

__global__ void blk_reset_kernel(BlkState *st, int B) {
  const int t = threadIdx.x;
  if (t < 3) st->slot[t] = kBlkNone;
  if (t == 0) { st->len = B; st->err = 0; }
  if (t < 64) {
    st->piv[t] = kBlkNone; st->mpiv[t] = 0; st->A[t] = 0; st->B0[t] = 0; st->Cp[t] = 0;
    st->rV[t] = 0; st->G[t] = 0;
  }
}

// C_r = x bits of row r at q_0..q_{B-1}; M = 0; base = original; T = parity = 0;
// pivot of step 0 by atomicMin
__global__ void __launch_bounds__(256)
blk_init_kernel(const uint64_t *__restrict__ RX, uint32_t rs, uint64_t nrows, uint32_t n, uint32_t k,
                const uint32_t *__restrict__ qubits, int B, uint64_t *__restrict__ C,
                uint64_t *__restrict__ M, int32_t *__restrict__ base, BlkState *st,
                uint32_t *__restrict__ err) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t c = 0;
  if (r < nrows) {
    uint32_t lastw = 0xFFFFFFFFu;
    uint64_t word = 0;
    for (int j = 0; j < B; ++j) {
      const uint32_t q = qubits[j];
      if (q >= n) { if (r == 0) atomicOr(err, kErrBadQubit); continue; }
      if ((q >> 6) != lastw) { lastw = q >> 6; word = RX[r * rs + lastw]; }
      c |= ((word >> (q & 63)) & 1ull) << j;
    }
    C[r] = c;
    M[r] = 0;
    base[r] = kBaseOrig;
  }
  const uint32_t ball = __ballot_sync(0xffffffffu, (c & 1ull) != 0);
  if ((threadIdx.x & 31) == 0 && r < nrows) {
    const uint64_t lo = 64ull * k, hi = 64ull * k + n, b0 = r;
    uint32_t m = ball;
    if (b0 + 32 > lo && b0 < hi && m) {
      if (b0 < lo) m &= ~0u << (uint32_t)(lo - b0);
      if (b0 + 32 > hi) m &= (uint32_t)((1ull << (hi - b0)) - 1);
      if (m) atomicMin(reinterpret_cast<long long *>(&st->slot[0]), (long long)(b0 + __ffs(m) - 1));
    }
  }
}

// symbolic step j: Cin -> Cout
__global__ void __launch_bounds__(256)
blk_step_kernel(uint64_t nrows, uint32_t n, uint32_t k, int j, int B, const uint64_t *__restrict__ Cin,
                uint64_t *__restrict__ Cout, uint64_t *__restrict__ M, int32_t *__restrict__ base,
                BlkState *st) {
  if (j >= st->len) return;
  const int64_t p = st->slot[j % 3];
  if (p == kBlkNone) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->len = j;
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->slot[(j + 2) % 3] = kBlkNone;
    st->piv[j] = p;
  }
  const int64_t pd = p - 64ll * k;
  const uint64_t cp = Cin[p];
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t c = 0;
  if (r < nrows) {
    c = Cin[r];
    if ((int64_t)r == p) {
      st->mpiv[j] = M[r];
      base[r] = kBasePivot + j;
      c = 0;
    } else if ((int64_t)r == pd) {
      c = cp;
      M[r] = 0;
      base[r] = j;
    } else if ((c >> j) & 1ull) {
      c ^= cp;
      M[r] |= 1ull << j;
    }
    Cout[r] = c;
  }
  if (j + 1 < B) {
    const uint32_t ball = __ballot_sync(0xffffffffu, ((c >> (j + 1)) & 1ull) != 0);
    if ((threadIdx.x & 31) == 0 && r < nrows) {
      const uint64_t lo = 64ull * k, hi = 64ull * k + n, b0 = r;
      uint32_t m = ball;
      if (b0 + 32 > lo && b0 < hi && m) {
        if (b0 < lo) m &= ~0u << (uint32_t)(lo - b0);
        if (b0 + 32 > hi) m &= (uint32_t)((1ull << (hi - b0)) - 1);
        if (m)
          atomicMin(reinterpret_cast<long long *>(&st->slot[(j + 1) % 3]), (long long)(b0 + __ffs(m) - 1));
      }
    }
  }
}

// pivot rows V_j and the per-word phase sums; one thread per column word u
__global__ void __launch_bounds__(128)
blk_vrows_kernel(const uint64_t *__restrict__ RX, const uint64_t *__restrict__ RZ, uint32_t rs,
                 uint32_t k, uint64_t *__restrict__ VX, uint64_t *__restrict__ VZ, BlkState *st) {
  const int L = st->len;
  __shared__ int sA[64], sB[64], sC[64];
  __shared__ unsigned long long sG[64];
  if (threadIdx.x < 64) { sA[threadIdx.x] = 0; sB[threadIdx.x] = 0; sC[threadIdx.x] = 0; sG[threadIdx.x] = 0; }
  __syncthreads();
  // every word of the padded row (u < rs): padding qubit words are zero in the
  // tableau and must come out zero from the V rows too
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < rs) {
    for (int j = 0; j < L; ++j) {
      const int64_t p = st->piv[j];
      const uint64_t x0 = RX[(uint64_t)p * rs + u], z0 = RZ[(uint64_t)p * rs + u];
      uint64_t vx = x0, vz = z0, m = st->mpiv[j];
      while (m) {
        const int s = __ffsll((long long)m) - 1;
        m &= m - 1;
        vx ^= VX[(uint64_t)s * rs + u];
        vz ^= VZ[(uint64_t)s * rs + u];
      }
      VX[(uint64_t)j * rs + u] = vx;
      VZ[(uint64_t)j * rs + u] = vz;
      const int a = __popcll(vx & vz), b = __popcll(x0 & z0), c = __popcll((vz ^ z0) & x0) & 1;
      if (a) atomicAdd(&sA[j], a);
      if (b) atomicAdd(&sB[j], b);
      if (c) atomicXor(&sC[j], 1);
    }
    for (int s = 0; s < L; ++s) {
      const uint64_t zs = VZ[(uint64_t)s * rs + u];
      uint64_t row = 0;
      for (int t = 0; t < L; ++t) row |= (uint64_t)(__popcll(zs & VX[(uint64_t)t * rs + u]) & 1) << t;
      if (row) atomicXor(&sG[s], (unsigned long long)row);
    }
  }
  __syncthreads();
  if (threadIdx.x < (uint32_t)L) {
    const int j = threadIdx.x;
    if (sA[j]) atomicAdd(&st->A[j], sA[j]);
    if (sB[j]) atomicAdd(&st->B0[j], sB[j]);
    if (sC[j]) atomicXor(&st->Cp[j], sC[j]);
    if (sG[j]) atomicXor(reinterpret_cast<unsigned long long *>(&st->G[j]), sG[j]);
  }
}

__device__ __forceinline__ int cross_pairs(const uint64_t *G, uint64_t m) {
  // parity of sum over s > t, both in m, of G[s] bit t
  int par = 0;
  uint64_t mm = m;
  while (mm) {
    const int s = __ffsll((long long)mm) - 1;
    mm &= mm - 1;
    par ^= __popcll(G[s] & m & ((1ull << s) - 1)) & 1;
  }
  return par;
}

// signs of V_j in step order (one thread)
__global__ void blk_signs_kernel(const uint64_t *__restrict__ S, BlkState *st, uint32_t *err) {
  if (threadIdx.x != 0) return;
  const int L = st->len;
  for (int j = 0; j < L; ++j) {
    const int64_t p = st->piv[j];
    const uint64_t m = st->mpiv[j];
    int e = 2 * (int)((S[p >> 6] >> (p & 63)) & 1u) + st->B0[j] - st->A[j] + 2 * st->Cp[j];
    uint64_t mm = m;
    while (mm) {
      const int s = __ffsll((long long)mm) - 1;
      mm &= mm - 1;
      e += 2 * st->rV[s] + st->A[s];
    }
    e += 2 * cross_pairs(st->G, m);
    e = m4(e);
    if (e & 1) atomicOr(err, kErrOddPhase);
    st->rV[j] = e >> 1;
  }
}

// phase 3: block = one chunk of kCW column words x a range of rows; warp per row
__global__ void __launch_bounds__(256)
blk_apply_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint32_t rs, uint64_t nrows,
                 const uint32_t *__restrict__ qubits, const uint64_t *__restrict__ VX,
                 const uint64_t *__restrict__ VZ, const uint64_t *__restrict__ M,
                 const int32_t *__restrict__ base, int32_t *__restrict__ Tp, const BlkState *st) {
  extern __shared__ ulonglong2 sv[];  // [64][kCW/2] x words, then [64][kCW/2] z words
  ulonglong2(*svx)[kCW / 2] = reinterpret_cast<ulonglong2(*)[kCW / 2]>(sv);
  ulonglong2(*svz)[kCW / 2] = reinterpret_cast<ulonglong2(*)[kCW / 2]>(sv + 64 * (kCW / 2));
  const int L = st->len;
  const uint32_t u0 = blockIdx.x * kCW;  // first column word of the chunk
  const uint32_t nv = min((uint32_t)kCW, rs - u0) / 2;
  for (int i = threadIdx.x; i < L * (kCW / 2); i += blockDim.x) {
    const int s = i / (kCW / 2), v = i % (kCW / 2);
    if ((uint32_t)v < nv) {
      svx[s][v] = *reinterpret_cast<const ulonglong2 *>(VX + (uint64_t)s * rs + u0 + 2 * v);
      svz[s][v] = *reinterpret_cast<const ulonglong2 *>(VZ + (uint64_t)s * rs + u0 + 2 * v);
    }
  }
  __syncthreads();
  if (L == 0) return;
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.y * (blockDim.x >> 5);
  const uint64_t w0 = (uint64_t)blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (uint64_t r = w0; r < nrows; r += warps) {
    const int32_t b = base[r];
    const uint64_t sr = M[r];
    if (b == kBaseOrig && sr == 0) continue;
    ulonglong2 *rx = reinterpret_cast<ulonglong2 *>(RX + r * rs + u0);
    ulonglong2 *rz = reinterpret_cast<ulonglong2 *>(RZ + r * rs + u0);
    if (b >= kBasePivot) {  // pivot row of step j: +-Z_q (sign set by blk_rows_kernel)
      const uint32_t q = qubits[b - kBasePivot];
      for (uint32_t v = lane; v < nv; v += 32) {
        rx[v] = make_ulonglong2(0, 0);
        const uint32_t w = u0 + 2 * v;
        ulonglong2 zz = make_ulonglong2(0, 0);
        if ((q >> 6) == w) zz.x = 1ull << (q & 63);
        if ((q >> 6) == w + 1) zz.y = 1ull << (q & 63);
        rz[v] = zz;
      }
      continue;
    }
    int t = 0, c = 0;
    for (uint32_t v = lane; v < nv; v += 32) {
      ulonglong2 xb, zb;
      if (b == kBaseOrig) { xb = rx[v]; zb = rz[v]; }
      else { xb = svx[b][v]; zb = svz[b][v]; }
      ulonglong2 xa = make_ulonglong2(0, 0), za = make_ulonglong2(0, 0);
      uint64_t m = sr;
      while (m) {
        const int s = __ffsll((long long)m) - 1;
        m &= m - 1;
        const ulonglong2 a = svx[s][v], bz = svz[s][v];
        xa.x ^= a.x; xa.y ^= a.y;
        za.x ^= bz.x; za.y ^= bz.y;
      }
      const ulonglong2 xf = make_ulonglong2(xb.x ^ xa.x, xb.y ^ xa.y);
      const ulonglong2 zf = make_ulonglong2(zb.x ^ za.x, zb.y ^ za.y);
      t += __popcll(xb.x & zb.x) + __popcll(xb.y & zb.y) - __popcll(xf.x & zf.x) - __popcll(xf.y & zf.y);
      c ^= (__popcll(za.x & xb.x) + __popcll(za.y & xb.y)) & 1;
      rx[v] = xf;
      rz[v] = zf;
    }
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, o);
      c ^= __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) Tp[(uint64_t)blockIdx.x * nrows + r] = t * 2 + (c & 1);
  }
}

// per row: new sign from the accumulated terms; pivot rows get their coin; record
__global__ void __launch_bounds__(256)
blk_rows_kernel(uint64_t *__restrict__ S, uint64_t nrows, const uint32_t *__restrict__ qubits,
                const uint64_t *__restrict__ M, const int32_t *__restrict__ base,
                const int32_t *__restrict__ Tp, uint32_t chunks, const BlkState *st, uint64_t m0,
                uint64_t seed,
                uint64_t shot, uint8_t *__restrict__ record, uint32_t *__restrict__ err) {
  const int L = st->len;
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < (uint64_t)L) {
    const uint32_t b = (uint32_t)(philox4x64_10(m0 + r, shot, 0, 0, seed, kCoinKey).v[0] & 1u);
    record[m0 + r] = (uint8_t)b;
  }
  uint64_t delta = 0;
  if (r < nrows && L > 0) {
    const int32_t b = base[r];
    const uint64_t sr = M[r];
    const uint64_t old = (S[r >> 6] >> (r & 63)) & 1u;
    uint64_t nb = old;
    if (b >= kBasePivot) {
      const int j = b - kBasePivot;
      nb = philox4x64_10(m0 + j, shot, 0, 0, seed, kCoinKey).v[0] & 1u;
    } else if (b != kBaseOrig || sr != 0) {
      const int rb = (b == kBaseOrig) ? (int)old : st->rV[b];
      int tsum = 0, csum = 0;
      for (uint32_t ch = 0; ch < chunks; ++ch) {
        const int32_t v = Tp[(uint64_t)ch * nrows + r];
        tsum += v >> 1;  // arithmetic shift: t
        csum ^= v & 1;
      }
      int e = 2 * rb + tsum + 2 * csum;
      uint64_t mm = sr;
      while (mm) {
        const int s = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        e += 2 * st->rV[s] + st->A[s];
      }
      e += 2 * cross_pairs(st->G, sr);
      e = m4(e);
      if (e & 1) atomicOr(err, kErrOddPhase);
      nb = (uint64_t)(e >> 1);
    }
    delta = (nb ^ old) << (r & 63);
  }
  // fold the sign changes of the 32 rows of this warp into one atomic
  for (int o = 16; o > 0; o >>= 1) delta |= __shfl_xor_sync(0xffffffffu, delta, o);
  if ((threadIdx.x & 31) == 0 && r < nrows && delta)
    atomicXor(reinterpret_cast<unsigned long long *>(&S[r >> 6]), delta);
}

static uint32_t blk_chunks(const Layout &L) { return (L.rs + kCW - 1) / kCW; }

size_t blocked_scratch_bytes(const Layout &L) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return 3 * al(L.nrows * 8) + al(L.nrows * 4) + al((size_t)blk_chunks(L) * L.nrows * 4) +
         2 * al(64ull * L.rs * 8) + al(sizeof(BlkState));
}

static uint64_t g_apply_attr_set = 0;

// Enqueues one block of up to 64 measurements; the number actually done is
// st->len (read by the host after the stream is synchronised).
cudaError_t launch_measure_block(const Dev &d, void *scratch, const uint32_t *qubits, int B,
                                 uint64_t m0, qs_key key, cudaStream_t s, int *launches,
                                 int32_t **len_dev) {
  const Layout &L = d.L;
  uint8_t *p = static_cast<uint8_t *>(scratch);
  auto take = [&](size_t bytes) { uint8_t *q = p; p += (bytes + 255) & ~size_t(255); return q; };
  uint64_t *C0 = reinterpret_cast<uint64_t *>(take(L.nrows * 8));
  uint64_t *C1 = reinterpret_cast<uint64_t *>(take(L.nrows * 8));
  uint64_t *M = reinterpret_cast<uint64_t *>(take(L.nrows * 8));
  int32_t *base = reinterpret_cast<int32_t *>(take(L.nrows * 4));
  const uint32_t chunks = blk_chunks(L);
  int32_t *Tp = reinterpret_cast<int32_t *>(take((size_t)chunks * L.nrows * 4));
  uint64_t *VX = reinterpret_cast<uint64_t *>(take(64ull * L.rs * 8));
  uint64_t *VZ = reinterpret_cast<uint64_t *>(take(64ull * L.rs * 8));
  BlkState *st = reinterpret_cast<BlkState *>(take(sizeof(BlkState)));
  const unsigned rb = (unsigned)((L.nrows + 255) / 256);
  blk_reset_kernel<<<1, 64, 0, s>>>(st, B);
  blk_init_kernel<<<rb, 256, 0, s>>>(d.RX, L.rs, L.nrows, L.n, L.k, qubits, B, C0, M, base, st,
                                     d.err);
  for (int j = 0; j < B; ++j)
    blk_step_kernel<<<rb, 256, 0, s>>>(L.nrows, L.n, L.k, j, B, (j & 1) ? C1 : C0,
                                       (j & 1) ? C0 : C1, M, base, st);
  blk_vrows_kernel<<<(L.rs + 127) / 128, 128, 0, s>>>(d.RX, d.RZ, L.rs, L.k, VX, VZ, st);
  blk_signs_kernel<<<1, 32, 0, s>>>(d.S, st, d.err);
  const size_t smem = 2ull * 64 * (kCW / 2) * sizeof(ulonglong2);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !((g_apply_attr_set >> dev) & 1u)) {
    cudaError_t e = cudaFuncSetAttribute(blk_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    g_apply_attr_set |= 1ull << dev;
  }
  const uint32_t rows_y = std::max<uint32_t>(1, (uint32_t)std::min<uint64_t>((uint64_t)d.sms * 8 / chunks + 1, L.nrows / 8 + 1));
  blk_apply_kernel<<<dim3(chunks, rows_y), 256, smem, s>>>(d.RX, d.RZ, L.rs, L.nrows, qubits, VX,
                                                           VZ, M, base, Tp, st);
  blk_rows_kernel<<<rb, 256, 0, s>>>(d.S, L.nrows, qubits, M, base, Tp, chunks, st, m0, key.seed,
                                     key.shot, d.record, d.err);
  if (launches) *launches += 6 + B;
  if (len_dev) *len_dev = &st->len;
  return cudaGetLastError();
}

}  // namespace qs
