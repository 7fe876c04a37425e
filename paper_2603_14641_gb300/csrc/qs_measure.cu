// Projective Z-measurement on the row-major tableau, CHP semantics (Sec. 2.5,
// "The CHP algorithm"), with every decision taken on the device (no host
// round trip per measurement, unlike Alg. 2's CopyFirstPivotToHost /
// CopySignBitToHost).
//
// Per measured qubit q (record index m), five launches:
//  1. gather:   column q of the x-part as a 2n-bit mask (warp ballots) and the
//               pivot p = smallest stabilizer row with x_pq = 1 (Sec. 2.5;
//               Alg. 5's "is some stabilizer anticommuting" test and Alg. 6's
//               first compacted pivot, as one ballot + atomicMin).
//  2. rowsum:   probabilistic case. Every row h != p, h != p - n with
//               x_hq = 1 becomes S_p * row_h. The pivot row is fixed, so rows
//               are independent (no loop-carried state, unlike Stim's CX
//               injection that Sec. 3.2 has to unfold). The new sign comes from
//               the mod-4 phase of the product, computed with popcounts:
//                 P_p P_h = (-1)^(r_p + r_h) i^(|x_p&z_p| + |x_h&z_h|
//                           + 2 z_p.x_h - |x'&z'|) sigma(x', z'),
//               x' = x_p ^ x_h, z' = z_p ^ z_h (|.| = popcount); this equals
//               AG's rowsum 2 r_h + 2 r_p + sum_j g(...) mod 4.
//  3. det partial: deterministic case. (-1)^m Z_q = prod of S_i over the
//               destabilizers D_i with x_iq = 1 (Sec. 2.5). The phase of a
//               product P_1 ... P_t of commuting Paulis is
//                 2 sum r + sum |x_a&z_a| + 2 sum_{a<b} z_a.x_b - |X&Z|,
//               and the cross term sum_{a<b} z_a.x_b (mod 2) is an exclusive
//               prefix-XOR of the z rows dotted with the x rows -- the same
//               kind of carried prefix the paper unfolds in Sec. 3.2 Eqs.
//               9-11. Because it is GF(2)-bilinear, chunks of rows can be
//               processed independently: chunk s yields its XOR totals
//               (X_s, Z_s) and its local cross parity.
//  4. det combine: cross parity += (X_s . Z_before(s)) over chunks in order,
//               checks X_total = 0 and Z_total = e_q (the product is +-Z_q).
//  5. finalize: probabilistic: D_{p-n} <- S_p, S_p <- (-1)^b Z_q with
//               b = Philox coin(seed, shot, m); deterministic: m from the
//               phase sum. Appends the outcome to the record.
// Kernels of the branch not taken exit on their first check.
#include <algorithm>
#include <climits>

#include "qs_internal.cuh"

namespace qs {

constexpr int64_t kNoPivot = LLONG_MAX;

__device__ __forceinline__ int mod4(int v) { return ((v % 4) + 4) % 4; }

__global__ void reset_meas_state_kernel(int64_t *mst) {
  if (threadIdx.x < kMeasStateWords) mst[threadIdx.x] = (threadIdx.x == kMsPivot) ? kNoPivot : 0;
}

cudaError_t launch_reset_meas_state(const Dev &d, cudaStream_t s) {
  reset_meas_state_kernel<<<1, 32, 0, s>>>(d.mst);
  return cudaGetLastError();
}

// 1. gather column q of the x-part; pivot by atomicMin
__global__ void __launch_bounds__(256)
gather_kernel(const uint64_t *__restrict__ RX, uint32_t rs, uint64_t nrows, uint32_t n, uint32_t k,
              const uint32_t *__restrict__ qubits, uint32_t qi, uint32_t *__restrict__ colx,
              int64_t *__restrict__ mst, uint32_t *__restrict__ err) {
  const uint32_t q = qubits[qi];
  if (q >= n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrBadQubit);
    return;
  }
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t bit = 0;
  if (r < nrows) bit = (uint32_t)(RX[r * rs + (q >> 6)] >> (q & 63)) & 1u;
  const uint32_t ball = __ballot_sync(0xffffffffu, bit);
  const int lane = threadIdx.x & 31;
  if (lane == 0 && r < nrows) {
    colx[r >> 5] = ball;
    // stabilizer rows are packed rows [64k, 64k + n)
    const uint64_t lo = 64ull * k, hi = 64ull * k + n;
    uint32_t m = ball;
    const uint64_t base = r;  // row of lane 0
    if (base + 32 > lo && base < hi && m) {
      if (base < lo) m &= ~0u << (uint32_t)(lo - base);
      if (base + 32 > hi) m &= (uint32_t)((1ull << (hi - base)) - 1);
      if (m) atomicMin(reinterpret_cast<long long *>(&mst[kMsPivot]), (long long)(base + __ffs(m) - 1));
    }
  }
}

// 2. rowsum of the pivot row into every anticommuting row (probabilistic case)
__global__ void __launch_bounds__(512)
rowsum_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint32_t rs, uint64_t nrows,
              uint32_t n, uint32_t k, uint64_t *__restrict__ S, const uint32_t *__restrict__ colx,
              const int64_t *__restrict__ mst, const uint32_t *__restrict__ qubits, uint32_t qi,
              uint32_t *__restrict__ err) {
  const uint32_t q = qubits[qi];
  if (q >= n) return;
  const int64_t p = mst[kMsPivot];
  if (p == kNoPivot) return;
  extern __shared__ uint64_t sm[];
  uint64_t *spx = sm, *spz = sm + rs;
  __shared__ int s_pxz[32];
  int pxz = 0;
  for (uint32_t u = threadIdx.x; u < rs; u += blockDim.x) {
    uint64_t x = RX[(uint64_t)p * rs + u], z = RZ[(uint64_t)p * rs + u];
    spx[u] = x; spz[u] = z;
    pxz += __popcll(x & z);
  }
  // block sum of |x_p & z_p|
  for (int o = 16; o > 0; o >>= 1) pxz += __shfl_xor_sync(0xffffffffu, pxz, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_pxz[warp] = pxz;
  __syncthreads();
  int tot_pxz = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot_pxz += s_pxz[w];
  const int rp = (int)((S[p >> 6] >> (p & 63)) & 1u);
  const int base = mod4(2 * rp + tot_pxz);
  const int64_t pd = p - 64ll * k;
  const uint32_t nvec = rs >> 1;  // 128-bit vectors per row (rs is a multiple of 4)
  const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const ulonglong2 *px2 = reinterpret_cast<const ulonglong2 *>(spx);
  const ulonglong2 *pz2 = reinterpret_cast<const ulonglong2 *>(spz);
  for (uint64_t r = gw; r < nrows; r += nw) {
    if (((colx[r >> 5] >> (r & 31)) & 1u) == 0 || (int64_t)r == p || (int64_t)r == pd) continue;
    ulonglong2 *rx = reinterpret_cast<ulonglong2 *>(RX + r * rs);
    ulonglong2 *rz = reinterpret_cast<ulonglong2 *>(RZ + r * rs);
    int acc = 0;
#pragma unroll 4
    for (uint32_t v = lane; v < nvec; v += 32) {
      ulonglong2 x = rx[v], z = rz[v], a = px2[v], c = pz2[v];
      ulonglong2 nx = make_ulonglong2(x.x ^ a.x, x.y ^ a.y);
      ulonglong2 nz = make_ulonglong2(z.x ^ c.x, z.y ^ c.y);
      acc += __popcll(x.x & z.x) + __popcll(x.y & z.y);
      acc += 2 * (__popcll(c.x & x.x) + __popcll(c.y & x.y));
      acc -= __popcll(nx.x & nz.x) + __popcll(nx.y & nz.y);
      rx[v] = nx;
      rz[v] = nz;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const int t = mod4(base + acc);
      if (t & 1) atomicOr(err, kErrOddPhase);
      if (t >> 1)
        atomicXor(reinterpret_cast<unsigned long long *>(&S[r >> 6]), 1ull << (r & 63));
    }
  }
}

// 3. deterministic case: per chunk of destabilizer rows, XOR totals of the
//    selected stabilizer rows, local cross parity and |x & z| + 2 r sums.
template <int UPT>
__global__ void __launch_bounds__(1024)
det_partial_kernel(const uint64_t *__restrict__ RX, const uint64_t *__restrict__ RZ, uint32_t rs,
                   uint32_t n, uint32_t k, const uint64_t *__restrict__ S,
                   const uint32_t *__restrict__ colx, const int64_t *__restrict__ mst,
                   const uint32_t *__restrict__ qubits, uint32_t qi, uint64_t *__restrict__ det_x,
                   uint64_t *__restrict__ det_z, int32_t *__restrict__ det_scal) {
  const uint32_t q = qubits[qi];
  if (q >= n) return;
  if (mst[kMsPivot] != kNoPivot) return;
  const uint32_t b = blockIdx.x;
  const uint32_t wpc = (k + gridDim.x - 1) / gridDim.x;  // 64-row words per chunk
  const uint32_t w0 = b * wpc, w1 = min(k, w0 + wpc);
  uint64_t px[UPT], pz[UPT];
#pragma unroll
  for (int j = 0; j < UPT; ++j) { px[j] = 0; pz[j] = 0; }
  uint64_t cross = 0;
  int cnt = 0, rsum = 0;
  const uint64_t *colx64 = reinterpret_cast<const uint64_t *>(colx);
  for (uint32_t w = w0; w < w1; ++w) {
    uint64_t m = colx64[w];  // destabilizer rows 64 w .. 64 w + 63
    if (threadIdx.x == 0) rsum += __popcll(m & S[k + w]);  // signs of S_i, i in this word
    while (m) {
      const int bit = __ffsll((long long)m) - 1;
      m &= m - 1;
      const uint64_t r = 64ull * k + 64ull * w + bit;  // stabilizer S_i, i = 64 w + bit
#pragma unroll
      for (int j = 0; j < UPT; ++j) {
        const uint32_t u = threadIdx.x + j * blockDim.x;
        if (u < k) {
          const uint64_t x = RX[r * rs + u], z = RZ[r * rs + u];
          cross ^= x & pz[j];
          cnt += __popcll(x & z);
          px[j] ^= x;
          pz[j] ^= z;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < UPT; ++j) {
    const uint32_t u = threadIdx.x + j * blockDim.x;
    if (u < k) {
      det_x[(uint64_t)b * rs + u] = px[j];
      det_z[(uint64_t)b * rs + u] = pz[j];
    }
  }
  int v = cnt + 2 * (__popcll(cross) & 1) + 2 * rsum;
  __shared__ int red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    det_scal[b] = mod4(t);
  }
}

// 4. combine chunks in order (one thread per word position u)
__global__ void __launch_bounds__(256)
det_combine_kernel(uint32_t rs, uint32_t n, uint32_t k, int64_t *mst,
                   const uint32_t *__restrict__ qubits, uint32_t qi,
                   const uint64_t *__restrict__ det_x, const uint64_t *__restrict__ det_z,
                   uint32_t nchunks, uint32_t *__restrict__ err) {
  const uint32_t q = qubits[qi];
  if (q >= n) return;
  if (mst[kMsPivot] != kNoPivot) return;
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t par = 0;
  bool bad = false;
  if (u < k) {
    uint64_t cross = 0, xb = 0, zb = 0;
    for (uint32_t b = 0; b < nchunks; ++b) {
      const uint64_t x = det_x[(uint64_t)b * rs + u], z = det_z[(uint64_t)b * rs + u];
      cross ^= x & zb;
      xb ^= x;
      zb ^= z;
    }
    par = __popcll(cross) & 1u;
    const uint64_t want = (u == (q >> 6)) ? (1ull << (q & 63)) : 0ull;
    bad = (xb != 0) || (zb != want);
  }
  const uint32_t bpar = __ballot_sync(0xffffffffu, par != 0);
  const uint32_t bbad = __ballot_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (__popc(bpar) & 1) atomicXor(reinterpret_cast<unsigned long long *>(&mst[kMsDetCross]), 1ull);
    if (bbad) atomicOr(err, kErrDetProduct);
  }
}

// 5. finalize the measurement and append the outcome
__global__ void __launch_bounds__(256)
finalize_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint32_t rs, uint32_t n,
                uint32_t k, uint64_t *__restrict__ S, int64_t *__restrict__ mst,
                const uint32_t *__restrict__ qubits, uint32_t qi, uint64_t midx, uint64_t seed,
                uint64_t shot, const int32_t *__restrict__ det_scal, uint32_t nchunks,
                uint8_t *__restrict__ record, uint8_t *__restrict__ kinds,
                uint32_t *__restrict__ err) {
  const uint32_t q = qubits[qi];
  const int64_t p = mst[kMsPivot];
  __syncthreads();
  if (q >= n) {
    if (threadIdx.x == 0) {
      record[midx] = 0;
      kinds[midx] = 0;
      mst[kMsPivot] = kNoPivot;
      mst[kMsDetCross] = 0;
    }
    return;
  }
  if (p != kNoPivot) {
    const int64_t pd = p - 64ll * k;
    for (uint32_t u = threadIdx.x; u < rs; u += blockDim.x) {
      const uint64_t x = RX[(uint64_t)p * rs + u], z = RZ[(uint64_t)p * rs + u];
      RX[(uint64_t)pd * rs + u] = x;  // D_{p-n} <- S_p
      RZ[(uint64_t)pd * rs + u] = z;
      RX[(uint64_t)p * rs + u] = 0;   // S_p <- (-1)^b Z_q
      RZ[(uint64_t)p * rs + u] = (u == (q >> 6)) ? (1ull << (q & 63)) : 0ull;
    }
    if (threadIdx.x == 0) {
      const uint32_t b = (uint32_t)(philox4x64_10(midx, shot, 0, 0, seed, kCoinKey).v[0] & 1u);
      const uint64_t sp = (S[p >> 6] >> (p & 63)) & 1u;
      S[pd >> 6] = (S[pd >> 6] & ~(1ull << (pd & 63))) | (sp << (pd & 63));
      S[p >> 6] = (S[p >> 6] & ~(1ull << (p & 63))) | ((uint64_t)b << (p & 63));
      record[midx] = (uint8_t)b;
      kinds[midx] = 1;
    }
  } else if (threadIdx.x == 0) {
    int t = 0;
    for (uint32_t b = 0; b < nchunks; ++b) t += det_scal[b];
    t += 2 * (int)(mst[kMsDetCross] & 1);
    t = mod4(t);
    if (t & 1) atomicOr(err, kErrOddPhase);
    record[midx] = (uint8_t)(t >> 1);
    kinds[midx] = 0;
  }
  if (threadIdx.x == 0) { mst[kMsPivot] = kNoPivot; mst[kMsDetCross] = 0; }
}

static std::atomic<uint64_t> g_rowsum_attr_set{0};

cudaError_t launch_gather(const Dev &d, const uint32_t *qubits, uint32_t i, cudaStream_t s) {
  const Layout &L = d.L;
  gather_kernel<<<(uint32_t)((L.nrows + 255) / 256), 256, 0, s>>>(d.RX, L.rs, L.nrows, L.n, L.k, qubits,
                                                                 i, d.colx, d.mst, d.err);
  return cudaGetLastError();
}

cudaError_t launch_measure_one(const Dev &d, const uint32_t *qubits, uint32_t i, uint64_t midx,
                               qs_key key, cudaStream_t s, int *launches) {
  const Layout &L = d.L;
  const uint32_t gblocks = (uint32_t)((L.nrows + 255) / 256);
  gather_kernel<<<gblocks, 256, 0, s>>>(d.RX, L.rs, L.nrows, L.n, L.k, qubits, i, d.colx, d.mst,
                                        d.err);
  const size_t smem = 2ull * L.rs * sizeof(uint64_t);
  if (smem > 48 * 1024) {
    cudaError_t ea = once_per_device(g_rowsum_attr_set, []() {
      return cudaFuncSetAttribute(rowsum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024);
    });
    if (ea != cudaSuccess) return ea;
  }
  const int sms = d.sms;
  // rows per warp ~ nrows / warps; at most 4 blocks of 512 per SM
  uint64_t want = (L.nrows + 15) / 16;
  uint32_t rblocks = (uint32_t)std::min<uint64_t>((uint64_t)sms * 4, std::max<uint64_t>(1, want));
  rowsum_kernel<<<rblocks, 512, smem, s>>>(d.RX, d.RZ, L.rs, L.nrows, L.n, L.k, d.S, d.colx,
                                           d.mst, qubits, i, d.err);
  const uint32_t nchunks = std::min<uint32_t>(kDetBlocks, L.k);
  uint32_t threads = std::min<uint32_t>(1024, (L.k + 31) / 32 * 32);
  uint32_t upt = (L.k + threads - 1) / threads;
  if (upt <= 1)
    det_partial_kernel<1><<<nchunks, threads, 0, s>>>(d.RX, d.RZ, L.rs, L.n, L.k, d.S, d.colx, d.mst,
                                                     qubits, i, d.det_x, d.det_z, d.det_scal);
  else if (upt <= 2)
    det_partial_kernel<2><<<nchunks, threads, 0, s>>>(d.RX, d.RZ, L.rs, L.n, L.k, d.S, d.colx, d.mst,
                                                     qubits, i, d.det_x, d.det_z, d.det_scal);
  else if (upt <= 4)
    det_partial_kernel<4><<<nchunks, threads, 0, s>>>(d.RX, d.RZ, L.rs, L.n, L.k, d.S, d.colx, d.mst,
                                                     qubits, i, d.det_x, d.det_z, d.det_scal);
  else
    det_partial_kernel<16><<<nchunks, threads, 0, s>>>(d.RX, d.RZ, L.rs, L.n, L.k, d.S, d.colx,
                                                      d.mst, qubits, i, d.det_x, d.det_z,
                                                      d.det_scal);
  det_combine_kernel<<<(L.k + 255) / 256, 256, 0, s>>>(L.rs, L.n, L.k, d.mst, qubits, i,
                                                       d.det_x, d.det_z, nchunks, d.err);
  finalize_kernel<<<1, 256, 0, s>>>(d.RX, d.RZ, L.rs, L.n, L.k, d.S, d.mst, qubits, i, midx,
                                    key.seed, key.shot, d.det_scal, nchunks, d.record, d.kinds, d.err);
  if (launches) *launches += 5;
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Pipelined measurement window: two launches per measurement.
//
// The same CHP steps as above, regrouped so that measurement j needs
//   U_j  update:   rowsum of the pivot into the anticommuting rows
//                  (probabilistic) or the deterministic-product chunks;
//   F_j  finalize: D_{p-n} <- S_p, S_p <- (-1)^b Z_q or the chunk combine,
//                  record; and, in the same launch, the gather and pivot
//                  search of measurement j + 1.
// F_j may gather while its block 0 rewrites rows p and p - n, because those are
// the only rows finalize changes and their new x bit at the next qubit is
// known: 0 for S_p (now +-Z_q) and, for D_{p-n}, the bit of the old pivot row,
// saved by U_j. The pivot search results alternate between two slots.
// ---------------------------------------------------------------------------
enum : int { kPivSlot0 = 0, kPivSlot1 = 1, kNextBit = 3 };

template <int UPT>
__global__ void __launch_bounds__(512)
meas_update_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint32_t rs,
                   uint64_t nrows, uint32_t n, uint32_t k, uint64_t *__restrict__ S,
                   const uint32_t *__restrict__ colx, int64_t *mst,
                   const uint32_t *__restrict__ qubits, uint32_t j, uint32_t has_next,
                   uint64_t *__restrict__ det_x, uint64_t *__restrict__ det_z,
                   int32_t *__restrict__ det_scal, uint32_t nchunks, uint32_t *__restrict__ err) {
  const int slot = j & 1;
  const int64_t p = mst[slot];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    mst[slot ^ 1] = kNoPivot;  // free for the pivot search of measurement j + 1
    if (p != kNoPivot && has_next) {
      const uint32_t q2 = qubits[j + 1];
      mst[kNextBit] = q2 < n ? (int64_t)((RX[(uint64_t)p * rs + (q2 >> 6)] >> (q2 & 63)) & 1u) : 0;
    }
  }
  const uint32_t q = qubits[j];
  if (q >= n) return;
  if (p != kNoPivot) {
    extern __shared__ uint64_t sm[];
    uint64_t *spx = sm, *spz = sm + rs;
    __shared__ int s_pxz[32];
    int pxz = 0;
    for (uint32_t u = threadIdx.x; u < rs; u += blockDim.x) {
      const uint64_t x = RX[(uint64_t)p * rs + u], z = RZ[(uint64_t)p * rs + u];
      spx[u] = x; spz[u] = z;
      pxz += __popcll(x & z);
    }
    for (int o = 16; o > 0; o >>= 1) pxz += __shfl_xor_sync(0xffffffffu, pxz, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_pxz[warp] = pxz;
    __syncthreads();
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_pxz[w];
    const int rp = (int)((S[p >> 6] >> (p & 63)) & 1u);
    const int base = mod4(2 * rp + tot);
    const int64_t pd = p - 64ll * k;
    const uint32_t nvec = rs >> 1;
    const uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const ulonglong2 *px2 = reinterpret_cast<const ulonglong2 *>(spx);
    const ulonglong2 *pz2 = reinterpret_cast<const ulonglong2 *>(spz);
    for (uint64_t r = gw; r < nrows; r += nw) {
      if (((colx[r >> 5] >> (r & 31)) & 1u) == 0 || (int64_t)r == p || (int64_t)r == pd) continue;
      ulonglong2 *rx = reinterpret_cast<ulonglong2 *>(RX + r * rs);
      ulonglong2 *rz = reinterpret_cast<ulonglong2 *>(RZ + r * rs);
      int acc = 0;
#pragma unroll 4
      for (uint32_t v = lane; v < nvec; v += 32) {
        const ulonglong2 x = rx[v], z = rz[v], a = px2[v], c = pz2[v];
        const ulonglong2 nx = make_ulonglong2(x.x ^ a.x, x.y ^ a.y);
        const ulonglong2 nz = make_ulonglong2(z.x ^ c.x, z.y ^ c.y);
        acc += __popcll(x.x & z.x) + __popcll(x.y & z.y);
        acc += 2 * (__popcll(c.x & x.x) + __popcll(c.y & x.y));
        acc -= __popcll(nx.x & nz.x) + __popcll(nx.y & nz.y);
        rx[v] = nx;
        rz[v] = nz;
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        const int t = mod4(base + acc);
        if (t & 1) atomicOr(err, kErrOddPhase);
        if (t >> 1) atomicXor(reinterpret_cast<unsigned long long *>(&S[r >> 6]), 1ull << (r & 63));
      }
    }
    return;
  }
  // deterministic: block b < nchunks folds the stabilizer rows S_i of its
  // chunk of destabilizer words (XOR totals, local cross parity, |x & z|, signs)
  const uint32_t b = blockIdx.x;
  if (b >= nchunks) return;
  const uint32_t wpc = (k + nchunks - 1) / nchunks;
  const uint32_t w0 = b * wpc, w1 = min(k, w0 + wpc);
  uint64_t px[UPT], pz[UPT];
#pragma unroll
  for (int t = 0; t < UPT; ++t) { px[t] = 0; pz[t] = 0; }
  uint64_t cross = 0;
  int cnt = 0, rsum = 0;
  const uint64_t *colx64 = reinterpret_cast<const uint64_t *>(colx);
  for (uint32_t w = w0; w < w1; ++w) {
    uint64_t m = colx64[w];
    if (threadIdx.x == 0) rsum += __popcll(m & S[k + w]);
    while (m) {
      const int bit = __ffsll((long long)m) - 1;
      m &= m - 1;
      const uint64_t r = 64ull * k + 64ull * w + bit;
#pragma unroll
      for (int t = 0; t < UPT; ++t) {
        const uint32_t u = threadIdx.x + t * blockDim.x;
        if (u < k) {
          const uint64_t x = RX[r * rs + u], z = RZ[r * rs + u];
          cross ^= x & pz[t];
          cnt += __popcll(x & z);
          px[t] ^= x;
          pz[t] ^= z;
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < UPT; ++t) {
    const uint32_t u = threadIdx.x + t * blockDim.x;
    if (u < k) {
      det_x[(uint64_t)b * rs + u] = px[t];
      det_z[(uint64_t)b * rs + u] = pz[t];
    }
  }
  int v = cnt + 2 * (__popcll(cross) & 1) + 2 * rsum;
  __shared__ int red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    det_scal[b] = mod4(t);
  }
}

__global__ void __launch_bounds__(256)
meas_finalize_gather_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint32_t rs,
                            uint64_t nrows, uint32_t n, uint32_t k, uint64_t *__restrict__ S,
                            uint32_t *__restrict__ colx, int64_t *mst,
                            const uint32_t *__restrict__ qubits, uint32_t j, uint32_t has_next,
                            uint64_t midx, uint64_t seed, uint64_t shot,
                            const uint64_t *__restrict__ det_x, const uint64_t *__restrict__ det_z,
                            const int32_t *__restrict__ det_scal, uint32_t nchunks,
                            uint8_t *__restrict__ record, uint8_t *__restrict__ kinds,
                            uint32_t *__restrict__ err) {
  const int slot = j & 1;
  const int64_t p = mst[slot];
  const uint32_t q = qubits[j];
  const bool prob = (q < n) && p != kNoPivot;
  const int64_t pd = prob ? p - 64ll * k : -1;
  // gather of measurement j + 1 (every block, one thread per packed row)
  if (has_next) {
    const uint32_t q2 = qubits[j + 1];
    if (q2 < n) {
      const int next_bit = (int)mst[kNextBit];
      const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
      uint32_t bit = 0;
      if (r < nrows) {
        if (prob && (int64_t)r == p) bit = 0;
        else if (prob && (int64_t)r == pd) bit = (uint32_t)next_bit;
        else bit = (uint32_t)(RX[r * rs + (q2 >> 6)] >> (q2 & 63)) & 1u;
      }
      const uint32_t ball = __ballot_sync(0xffffffffu, bit);
      if ((threadIdx.x & 31) == 0 && r < nrows) {
        colx[r >> 5] = ball;
        const uint64_t lo = 64ull * k, hi = 64ull * k + n, base = r;
        uint32_t m = ball;
        if (base + 32 > lo && base < hi && m) {
          if (base < lo) m &= ~0u << (uint32_t)(lo - base);
          if (base + 32 > hi) m &= (uint32_t)((1ull << (hi - base)) - 1);
          if (m)
            atomicMin(reinterpret_cast<long long *>(&mst[slot ^ 1]), (long long)(base + __ffs(m) - 1));
        }
      }
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicOr(err, kErrBadQubit);
    }
  }
  if (blockIdx.x != 0) return;
  // finalize measurement j (block 0)
  if (q >= n) {
    if (threadIdx.x == 0) { record[midx] = 0; kinds[midx] = 0; atomicOr(err, kErrBadQubit); }
    return;
  }
  if (prob) {
    for (uint32_t u = threadIdx.x; u < rs; u += blockDim.x) {
      const uint64_t x = RX[(uint64_t)p * rs + u], z = RZ[(uint64_t)p * rs + u];
      RX[(uint64_t)pd * rs + u] = x;  // D_{p-n} <- S_p
      RZ[(uint64_t)pd * rs + u] = z;
      RX[(uint64_t)p * rs + u] = 0;   // S_p <- (-1)^b Z_q
      RZ[(uint64_t)p * rs + u] = (u == (q >> 6)) ? (1ull << (q & 63)) : 0ull;
    }
    if (threadIdx.x == 0) {
      const uint32_t b = (uint32_t)(philox4x64_10(midx, shot, 0, 0, seed, kCoinKey).v[0] & 1u);
      const uint64_t sp = (S[p >> 6] >> (p & 63)) & 1u;
      S[pd >> 6] = (S[pd >> 6] & ~(1ull << (pd & 63))) | (sp << (pd & 63));
      S[p >> 6] = (S[p >> 6] & ~(1ull << (p & 63))) | ((uint64_t)b << (p & 63));
      record[midx] = (uint8_t)b;
      kinds[midx] = 1;
    }
    return;
  }
  // deterministic: combine the chunk totals in order (cross += X_s . Z_before(s))
  __shared__ int s_par, s_bad;
  if (threadIdx.x == 0) { s_par = 0; s_bad = 0; }
  __syncthreads();
  for (uint32_t u = threadIdx.x; u < k; u += blockDim.x) {
    uint64_t cross = 0, xb = 0, zb = 0;
    for (uint32_t c = 0; c < nchunks; ++c) {
      const uint64_t x = det_x[(uint64_t)c * rs + u], z = det_z[(uint64_t)c * rs + u];
      cross ^= x & zb;
      xb ^= x;
      zb ^= z;
    }
    const uint64_t want = (u == (q >> 6)) ? (1ull << (q & 63)) : 0ull;
    if (__popcll(cross) & 1) atomicXor(&s_par, 1);
    if (xb != 0 || zb != want) atomicOr(&s_bad, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 2 * s_par;
    for (uint32_t c = 0; c < nchunks; ++c) t += det_scal[c];
    t = mod4(t);
    if (t & 1) atomicOr(err, kErrOddPhase);
    if (s_bad) atomicOr(err, kErrDetProduct);
    record[midx] = (uint8_t)(t >> 1);
    kinds[midx] = 0;
  }
}

static std::atomic<uint64_t> g_update_attr_set{0};

template <int UPT>
static void launch_update_t(const Dev &d, uint32_t rblocks, size_t smem, const uint32_t *qubits,
                            uint32_t j, uint32_t has_next, uint32_t nchunks, cudaStream_t s) {
  const Layout &L = d.L;
  meas_update_kernel<UPT><<<rblocks, 512, smem, s>>>(d.RX, d.RZ, L.rs, L.nrows, L.n, L.k, d.S,
                                                     d.colx, d.mst, qubits, j, has_next, d.det_x,
                                                     d.det_z, d.det_scal, nchunks, d.err);
}

bool measure_window_supported(const Layout &L) { return L.k <= 512u * 16u; }

cudaError_t launch_measure_window(const Dev &d, const uint32_t *qubits, uint32_t count,
                                  uint64_t m0, qs_key key, cudaStream_t s, int *launches) {
  if (count == 0) return cudaSuccess;
  const Layout &L = d.L;
  const size_t smem = 2ull * L.rs * sizeof(uint64_t);
  cudaError_t ea = once_per_device(g_update_attr_set, []() {
    for (cudaError_t e : {cudaFuncSetAttribute(meas_update_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                          cudaFuncSetAttribute(meas_update_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                          cudaFuncSetAttribute(meas_update_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                          cudaFuncSetAttribute(meas_update_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                          cudaFuncSetAttribute(meas_update_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)})
      if (e != cudaSuccess) return e;
    return cudaSuccess;
  });
  if (ea != cudaSuccess) return ea;
  const uint64_t want = (L.nrows + 15) / 16;
  const uint32_t rblocks = (uint32_t)std::min<uint64_t>((uint64_t)d.sms * 4, std::max<uint64_t>(1, want));
  const uint32_t nchunks = std::min<uint32_t>(std::min<uint32_t>(kDetBlocks, L.k), rblocks);
  const uint32_t upt = (L.k + 511) / 512;
  const uint32_t gblocks = (uint32_t)((L.nrows + 255) / 256);
  reset_meas_state_kernel<<<1, 32, 0, s>>>(d.mst);
  gather_kernel<<<gblocks, 256, 0, s>>>(d.RX, L.rs, L.nrows, L.n, L.k, qubits, 0, d.colx, d.mst,
                                        d.err);
  int l = 2;
  for (uint32_t j = 0; j < count; ++j) {
    const uint32_t has_next = j + 1 < count;
    if (upt <= 1) launch_update_t<1>(d, rblocks, smem, qubits, j, has_next, nchunks, s);
    else if (upt <= 2) launch_update_t<2>(d, rblocks, smem, qubits, j, has_next, nchunks, s);
    else if (upt <= 4) launch_update_t<4>(d, rblocks, smem, qubits, j, has_next, nchunks, s);
    else if (upt <= 8) launch_update_t<8>(d, rblocks, smem, qubits, j, has_next, nchunks, s);
    else launch_update_t<16>(d, rblocks, smem, qubits, j, has_next, nchunks, s);
    meas_finalize_gather_kernel<<<gblocks, 256, 0, s>>>(
        d.RX, d.RZ, L.rs, L.nrows, L.n, L.k, d.S, d.colx, d.mst, qubits, j, has_next, m0 + j,
        key.seed, key.shot, d.det_x, d.det_z, d.det_scal, nchunks, d.record, d.kinds, d.err);
    l += 2;
  }
  if (launches) *launches += l;
  return cudaGetLastError();
}

}  // namespace qs
