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
constexpr int kCW = 32;               // column words per phase-3 chunk
// windows of the lazy symbolic pass: stabilizer rows per window = threads of its
// CTA. 256 took the pass from 30.9 to 23.8 ms per step on the 10k workload and
// from 0.56 to 0.45 ms at 180k against 1,024 (512: 24.3 and 0.47 ms): a step
// waits on barriers of 8 warps instead of 32.
constexpr int kLazyLog2 = 8;
constexpr int kLazyThreads = 1 << kLazyLog2;
constexpr uint32_t kLazyMaxWindows = (1u << 20) >> kLazyLog2;  // n <= 2^20

struct BlkState {
  int64_t slot[3];     // pivot search results, rotating
  int32_t len;         // steps completed in this block
  uint32_t ntouched;   // rows the block changes (entries of the apply pass's row list)
  uint32_t i0;         // first measurement of the block within its window
  int32_t B;           // measurements the block attempts (0 past the window's end)
  uint32_t cursor;     // next measurement of the window: read by the next block's reset
  int64_t piv[64];     // pivot row of each step
  uint64_t mpiv[64];   // steps that targeted the pivot row before it became pivot
  int32_t A[64];       // |x_V & z_V| mod 4 (summed over words)
  int32_t B0[64];      // |x & z| of the original pivot row
  int32_t Cp[64];      // parity of (z_V ^ z_orig) . x_orig
  int32_t rV[64];      // sign bit of V_j
  uint64_t G[64];      // G[s] bit t = parity(z_{V_s} . x_{V_t})
  uint64_t cpiv[64];   // C of the pivot row at its step (lazy symbolic pass)
  uint32_t err;
  uint32_t pad2;
  uint64_t win_or[4096];  // OR of C over each window of stabilizer rows (lazy pass)
};

__device__ __forceinline__ int m4(int v) { return ((v % 4) + 4) % 4; }

// the block starts where the previous block of the window stopped (st->cursor),
// so the host can enqueue several blocks before it reads how far they got
__global__ void blk_reset_kernel(BlkState *st, uint32_t count, uint32_t nwin) {
  const int t = threadIdx.x;
  const uint32_t i0 = st->cursor;
  const int B = i0 < count ? (int)min(64u, count - i0) : 0;
  if (t < 3) st->slot[t] = kBlkNone;
  if (t == 0) { st->len = B; st->err = 0; st->ntouched = 0; st->i0 = i0; st->B = B; }
  if (t < 64) {
    st->piv[t] = kBlkNone; st->mpiv[t] = 0; st->A[t] = 0; st->B0[t] = 0; st->Cp[t] = 0;
    st->rV[t] = 0; st->G[t] = 0;
  }
  for (uint32_t w = t; w < nwin; w += blockDim.x) st->win_or[w] = 0;
}

// C_r = x bits of row r at q_0..q_{B-1}; M = 0; base = original; T = parity = 0;
// pivot of step 0 by atomicMin
__global__ void __launch_bounds__(256)
blk_init_kernel(const uint64_t *__restrict__ RX, uint32_t rs, uint64_t nrows, uint32_t n, uint32_t k,
                const uint32_t *__restrict__ window, uint64_t *__restrict__ C,
                uint64_t *__restrict__ M, int32_t *__restrict__ base, BlkState *st,
                uint32_t *__restrict__ err) {
  const int B = st->B;
  const uint32_t *qubits = window + st->i0;
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
  {
    // OR of C over this warp's 32 rows (in one window of stabilizer rows: the
    // stabilizer half starts at 64 k, a multiple of 32)
    uint64_t o = (r >= 64ull * k && r < 64ull * k + n) ? c : 0;
    for (int d = 16; d > 0; d >>= 1) o |= __shfl_xor_sync(0xffffffffu, o, d);
    if ((threadIdx.x & 31) == 0 && o)
      atomicOr(reinterpret_cast<unsigned long long *>(&st->win_or[(r - 64ull * k) >> kLazyLog2]), o);
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
blk_step_kernel(uint64_t nrows, uint32_t n, uint32_t k, int j, const uint64_t *__restrict__ Cin,
                uint64_t *__restrict__ Cout, uint64_t *__restrict__ M, int32_t *__restrict__ base,
                BlkState *st) {
  if (j >= st->len) return;
  const int B = st->B;
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

// Lazy symbolic pass in one CTA, for any n: only the pivot sequence
// (p_j, C_{p_j}) is needed here (blk_replay_kernel then derives every row's M_r
// and base_r from it), and the pivot of step j is the first stabilizer row, in
// index order, whose current C has bit j. So the stabilizer rows are scanned in
// windows of kLazyThreads (one row per thread), in order, and a window's rows are
// brought up to step j (replaying steps a_w..j-1 on them: the pivot row of a
// step becomes 0, a row with bit s set takes ^= C_{p_s}) only when it can hold
// bit j. That is decided from U_w, an upper bound on the OR of the window's C:
// exact when the window was last replayed, then grown by C_{p_s} for every
// step s whose bit U_w has (a row that takes C_{p_s} had bit s). In a dense
// state the pivots come from the first nonzero window, so a step costs one
// window and one barrier; rows far from the front are never read. Rows of
// replayed windows live in a working copy (W, the second C buffer); C0 stays
// intact for the replay kernel.

__device__ __forceinline__ uint64_t lazy_bound(uint64_t u, int a, int j, const uint64_t *cp) {
  for (int s = a; s < j; ++s)
    if ((u >> s) & 1ull) u |= cp[s];
  return u;
}

__global__ void __launch_bounds__(kLazyThreads)
blk_lazy_symbolic_kernel(uint32_t n, uint32_t k, const uint64_t *__restrict__ C0,
                         uint64_t *__restrict__ W, BlkState *st) {
  const int B = st->B;
  __shared__ uint64_t su[kLazyMaxWindows];   // U_w
  __shared__ uint8_t sa[kLazyMaxWindows];    // a_w: steps replayed on the window's rows
  __shared__ uint8_t sinit[kLazyMaxWindows]; // rows already in the working copy
  __shared__ int32_t spiv[64];               // stabilizer index of each step's pivot
  __shared__ uint64_t scp[64];               // its C at that step
  __shared__ uint32_t srow[2][32];           // per warp: first row with bit j (or ~0u)
  __shared__ uint64_t sval[2][32], sor[2][32];
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t nwin = (n + kLazyThreads - 1) >> kLazyLog2;
  const uint64_t lo = 64ull * k;
  for (uint32_t w = tid; w < nwin; w += kLazyThreads) {
    su[w] = st->win_or[w];
    sa[w] = 0;
    sinit[w] = 0;
  }
  if (tid < 64) {  // slots of warps the block does not have stay empty
    srow[tid >> 5][tid & 31] = 0xFFFFFFFFu;
    sval[tid >> 5][tid & 31] = 0;
    sor[tid >> 5][tid & 31] = 0;
  }
  __syncthreads();
  uint32_t front = 0;  // first window that may hold a nonzero row (uniform)
  while (front < nwin && su[front] == 0) ++front;
  int len = B, par = 0;
  uint32_t cw = 0xFFFFFFFFu;  // window whose row this thread holds in cc
  uint64_t cc = 0;
  for (int j = 0; j < B; ++j) {
    uint32_t hit = 0xFFFFFFFFu;
    uint64_t hitc = 0;
    for (uint32_t w = front; w < nwin; ++w) {
      const int a = sa[w];
      if (!((lazy_bound(su[w], a, j, scp) >> j) & 1ull)) continue;  // no row can have bit j
      // bring row kLazyThreads w + tid up to step j
      const uint32_t i = w * kLazyThreads + tid;
      uint64_t c = 0;
      if (i < n) {
        if (cw == w) c = cc;
        else c = sinit[w] ? W[lo + i] : C0[lo + i];
        for (int s2 = a; s2 < j; ++s2) {
          if ((int32_t)i == spiv[s2]) c = 0;
          else if ((c >> s2) & 1ull) c ^= scp[s2];
        }
        if (cw != w && cw != 0xFFFFFFFFu) W[lo + cw * kLazyThreads + tid] = cc;  // evict the held row
        cw = w;
        cc = c;
      }
      const bool has = i < n && ((c >> j) & 1ull);
      const uint32_t ball = __ballot_sync(0xffffffffu, has);
      const uint32_t first = ball ? (uint32_t)(__ffs(ball) - 1) : 32u;
      const uint64_t fc = __shfl_sync(0xffffffffu, c, first & 31);
      uint64_t o = c;
      for (int d = 16; d > 0; d >>= 1) o |= __shfl_xor_sync(0xffffffffu, o, d);
      if (lane == 0) {
        srow[par][warp] = ball ? warp * 32 + first : 0xFFFFFFFFu;
        sval[par][warp] = fc;
        sor[par][warp] = o;
      }
      __syncthreads();
      // every warp reduces the 32 per-warp slots lane-parallel (lane v reads slot v)
      const uint32_t rv = srow[par][lane];
      const uint64_t vv = sval[par][lane], ov = sor[par][lane];
      const uint32_t best = __reduce_min_sync(0xffffffffu, rv);
      const uint32_t bl = __ffs(__ballot_sync(0xffffffffu, rv == best)) - 1;
      const uint64_t bc = __shfl_sync(0xffffffffu, vv, bl);
      const uint64_t wor = ((uint64_t)__reduce_or_sync(0xffffffffu, (uint32_t)(ov >> 32)) << 32) |
                           __reduce_or_sync(0xffffffffu, (uint32_t)ov);
      par ^= 1;
      if (tid == 0) {
        su[w] = wor;
        sa[w] = (uint8_t)j;
        sinit[w] = 1;
      }
      if (best != 0xFFFFFFFFu) {
        hit = w * kLazyThreads + best;
        hitc = bc;
        break;
      }
    }
    if (hit == 0xFFFFFFFFu) { len = j; break; }  // deterministic: the block ends before step j
    if (tid == 0) {
      spiv[j] = (int32_t)hit;
      scp[j] = hitc;
      st->piv[j] = (int64_t)(lo + hit);
      st->cpiv[j] = hitc;
    }
    __syncthreads();  // su/sa/sinit and the new pivot are visible to every thread
  }
  if (tid == 0) st->len = len;
}

__global__ void __launch_bounds__(256)
blk_replay_kernel(uint64_t nrows, uint32_t k, const uint64_t *__restrict__ C0,
                  uint64_t *__restrict__ M, int32_t *__restrict__ base, BlkState *st) {
  __shared__ int64_t sp[64];
  __shared__ uint64_t sc[64];
  const int L = st->len;
  if (threadIdx.x < 64 && (int)threadIdx.x < L) {
    sp[threadIdx.x] = st->piv[threadIdx.x];
    sc[threadIdx.x] = st->cpiv[threadIdx.x];
  }
  __syncthreads();
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int64_t lo = 64ll * k;
  uint64_t c = C0[r], m = 0;
  int32_t b = kBaseOrig;
  for (int j = 0; j < L; ++j) {
    const int64_t p = sp[j];
    if ((int64_t)r == p) {
      st->mpiv[j] = m;
      b = kBasePivot + j;
      c = 0;
    } else if ((int64_t)r == p - lo) {
      c = sc[j];
      m = 0;
      b = j;
    } else if ((c >> j) & 1ull) {
      c ^= sc[j];
      m |= 1ull << j;
    }
  }
  M[r] = m;
  base[r] = b;
}

// pivot rows V_j and their phase sums for one chunk of 32 column words.
// V_j is the product of the original pivot rows p_s over a set E_j of steps:
// E_j = {j} xor (xor of E_s over the steps s that targeted p_j before step j),
// built by one warp in step order; every V_j of the chunk is then independent.
// Lane = column word; warp w takes steps w, w + 32; four blocks per chunk
// share the pairwise parities G.
constexpr int kVrowThreads = 1024;
constexpr int kVrowSplit = 4;  // blocks per chunk; block y computes G rows 16 y .. 16 y + 15
constexpr size_t kVrowSmem = 4ull * 64 * 32 * sizeof(uint64_t);  // original and V rows, x and z

__global__ void __launch_bounds__(kVrowThreads)
blk_vrows_kernel(const uint64_t *__restrict__ RX, const uint64_t *__restrict__ RZ, uint32_t rs,
                 uint64_t *__restrict__ VX, uint64_t *__restrict__ VZ, BlkState *st) {
  extern __shared__ uint64_t vsm[];
  uint64_t(*ox)[32] = reinterpret_cast<uint64_t(*)[32]>(vsm);
  uint64_t(*oz)[32] = reinterpret_cast<uint64_t(*)[32]>(vsm + 64 * 32);
  uint64_t(*vx)[32] = reinterpret_cast<uint64_t(*)[32]>(vsm + 2 * 64 * 32);
  uint64_t(*vz)[32] = reinterpret_cast<uint64_t(*)[32]>(vsm + 3 * 64 * 32);
  __shared__ uint64_t sE[64];
  const int L = st->len;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool lead = blockIdx.y == 0;  // writes the V rows and the per-step sums
  // every word of the padded row (u < rs): padding qubit words are zero in the
  // tableau and come out zero in the V rows too
  const uint32_t u = blockIdx.x * 32 + lane;
  const bool in = u < rs;
  for (int j = w; j < L; j += nw) {
    const uint64_t p = (uint64_t)st->piv[j];
    ox[j][lane] = in ? RX[p * rs + u] : 0;
    oz[j][lane] = in ? RZ[p * rs + u] : 0;
  }
  if (w == 0) {
    // E_j = {j} + sum of E_s over the steps s < j that targeted p_j (m_j), one
    // step after another: lane l keeps E_l and E_{l+32} in registers and each
    // step is one XOR reduction over the warp; the masks are loaded once
    const uint64_t mlo = lane < L ? st->mpiv[lane] : 0, mhi = lane + 32 < L ? st->mpiv[lane + 32] : 0;
    uint64_t elo = 0, ehi = 0;
    for (int j = 0; j < L; ++j) {
      const uint64_t m = __shfl_sync(0xffffffffu, j < 32 ? mlo : mhi, j & 31);  // only steps before j
      const uint64_t acc = (((m >> lane) & 1u) ? elo : 0) ^ (((m >> (lane + 32)) & 1u) ? ehi : 0);
      const uint64_t ej = (((uint64_t)__reduce_xor_sync(0xffffffffu, (uint32_t)(acc >> 32)) << 32) |
                           __reduce_xor_sync(0xffffffffu, (uint32_t)acc)) ^ (1ull << j);
      if (lane == (j & 31)) {
        if (j < 32) elo = ej;
        else ehi = ej;
      }
    }
    if (lane < L) sE[lane] = elo;
    if (lane + 32 < L) sE[lane + 32] = ehi;
  }
  __syncthreads();
  // every block builds all V rows of its chunk (G needs them); the lead block
  // also stores them and adds the per-step popcount sums
  for (int j = w; j < L; j += nw) {
    const uint64_t x0 = ox[j][lane], z0 = oz[j][lane];
    uint64_t ax = x0, az = z0, e = sE[j] & ~(1ull << j);
    while (e) {
      const int s2 = __ffsll((long long)e) - 1;
      e &= e - 1;
      ax ^= ox[s2][lane];
      az ^= oz[s2][lane];
    }
    vx[j][lane] = ax;
    vz[j][lane] = az;
    if (!lead) continue;
    if (in) {
      VX[(uint64_t)j * rs + u] = ax;
      VZ[(uint64_t)j * rs + u] = az;
    }
    int a = __popcll(ax & az), b = __popcll(x0 & z0);
    const uint32_t c = __ballot_sync(0xffffffffu, __popcll((az ^ z0) & x0) & 1);
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      if (a) atomicAdd(&st->A[j], a);
      if (b) atomicAdd(&st->B0[j], b);
      if (__popc(c) & 1) atomicXor(&st->Cp[j], 1);
    }
  }
  __syncthreads();
  // G[s] bit t = parity of z_{V_s} . x_{V_t} over the chunk: block y takes
  // s = 16 y + w / 2, each warp half of the t range
  const int sg = 16 * (int)blockIdx.y + (w >> 1), t0 = 32 * (w & 1);
  if (sg < L) {
    const uint64_t zs = vz[sg][lane];
    uint64_t row = 0;
    for (int t = t0; t < t0 + 32 && t < L; ++t) {
      const uint32_t bal = __ballot_sync(0xffffffffu, __popcll(zs & vx[t][lane]) & 1);
      row |= (uint64_t)(__popc(bal) & 1) << t;
    }
    if (lane == 0 && row) atomicXor(reinterpret_cast<unsigned long long *>(&st->G[sg]), row);
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

// signs of V_j. The phase exponent of step j is
//   e_j = 2 r(p_j) + B0_j - A_j + 2 Cp_j + sum_{s in m_j} (2 rV_s + A_s) + 2 cross(m_j)
// (mod 4); everything but the 2 rV_s terms is independent of the other steps and
// is computed by one thread per step, then one thread resolves the signs in
// step order: rV_j = (e'_j >> 1) ^ parity(m_j & {s : rV_s = 1}).
__global__ void __launch_bounds__(64) blk_signs_kernel(const uint64_t *__restrict__ S, BlkState *st,
                                                       uint32_t *err) {
  __shared__ int sb[64], sA[64];
  __shared__ uint64_t sm[64], sG[64];
  const int L = st->len, j = threadIdx.x;
  if (j < L) {
    sm[j] = st->mpiv[j];
    sA[j] = st->A[j];
    sG[j] = st->G[j];
  }
  __syncthreads();
  if (j < L) {
    const int64_t p = st->piv[j];
    const uint64_t m = sm[j];
    int e = 2 * (int)((S[p >> 6] >> (p & 63)) & 1u) + st->B0[j] - sA[j] + 2 * st->Cp[j];
    uint64_t mm = m;
    while (mm) {
      const int s = __ffsll((long long)mm) - 1;
      mm &= mm - 1;
      e += sA[s];
    }
    e += 2 * cross_pairs(sG, m);
    sb[j] = m4(e);
  }
  __syncthreads();
  if (j == 0) {
    uint64_t R = 0;
    for (int i = 0; i < L; ++i) {
      const int e = sb[i];
      if (e & 1) atomicOr(err, kErrOddPhase);
      const int rv = (e >> 1) ^ (__popcll(sm[i] & R) & 1);
      R |= (uint64_t)rv << i;
    }
    for (int i = 0; i < L; ++i) st->rV[i] = (int)((R >> i) & 1u);
  }
}

// phase 3: block = one chunk of kCW (32) column words x a range of rows.
// The XOR of any subset of the 64 V rows is assembled from tables of XOR
// combinations of consecutive steps (the "Four Russians" method), built once
// per block: T[g][c] = XOR of V[first step of g + b] over the bits b of c. A
// warp handles one row (lane = column word, x and z side by side in one
// 16-byte entry, 512 bytes per entry over the warp); a row segment is 256
// contiguous bytes of each matrix, the shortest that keeps HBM fully
// efficient. Each warp keeps the next two rows' loads in flight while it
// works on the current one; the row loop is unrolled by three so the
// in-flight rows rotate through registers without copies.
//
// The tables live in two memories of the SM. Steps 0..43 use shared memory:
// seven groups of 6 steps and one of 2 (452 entries, 226 KB). Steps 44..63
// use tensor memory (TMEM, 512 columns x 128 lanes of 32 bits): four groups
// of 5 steps. TMEM lane l of each 32-lane quarter holds column word l of the
// chunk and every quarter holds the same four tables (a warp reads only the
// lanes of its quarter, warp mod 4), so an entry is 4 columns (x lo, x hi,
// z lo, z hi) and group t, pattern p sits at columns 128 t + 4 p. A row costs
// 8 shared-memory lookups (32 wavefronts; 13 lookups and 52 wavefronts with
// 5-step groups in shared memory alone, which bounded the pass on the
// shared-memory pipe) and 4 TMEM loads on the tensor-memory read path.
constexpr int kEntryBytes = kCW * 16;   // 512

struct ApplyRow {
  uint32_t r;
  int32_t b;
  uint32_t lo, hi;  // M_r
  uint2 x, z;       // this lane's word of x and z, as 32-bit halves
};

// row, pattern M_r and base_r of a row the block changes (one stage ahead of
// its words): entry j of the row list, or row = nrows past its end
struct ApplyMeta {
  uint32_t r;
  int32_t b;
  uint32_t lo, hi;
};

__device__ __forceinline__ void apply_meta(ApplyMeta &m, uint32_t j, uint32_t cnt, uint32_t nrows,
                                           const uint4 *list) {
  m.r = nrows;
  m.b = kBaseOrig;
  m.lo = m.hi = 0;
  if (j < cnt) {
    const uint4 e = __ldg(list + j);
    m.r = e.x;
    m.b = (int32_t)e.y;
    m.lo = e.z;
    m.hi = e.w;
  }
}

// the row list: every row the block changes (a step targeted it, or its base
// changed: replaced destabilizers and the new pivots) with its pattern and
// base, in groups of consecutive rows (one atomic per warp). Rows left alone
// (M_r = 0, original base: e.g. the +-Z_q pivot rows of earlier blocks) are
// neither listed, read nor written.
__global__ void __launch_bounds__(256)
blk_list_kernel(uint64_t nrows, const uint64_t *__restrict__ M, const int32_t *__restrict__ base,
                uint4 *__restrict__ list, BlkState *st) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t m = 0;
  int32_t b = kBaseOrig;
  if (r < nrows) {
    m = M[r];
    b = base[r];
  }
  const bool touched = r < nrows && (b != kBaseOrig || m != 0);
  const uint32_t ball = __ballot_sync(0xffffffffu, touched);
  const uint32_t lane = threadIdx.x & 31;
  uint32_t at = 0;
  if (lane == 0 && ball) at = atomicAdd(&st->ntouched, (uint32_t)__popc(ball));
  at = __shfl_sync(0xffffffffu, at, 0);
  if (touched)
    list[at + __popc(ball & ((1u << lane) - 1))] =
        make_uint4((uint32_t)r, (uint32_t)b, (uint32_t)m, (uint32_t)(m >> 32));
}

// the row's words, fetched only when the row changes: a row that no step
// targeted and that kept its original base (M_r = 0, base_r original; e.g.
// the +-Z_q pivot rows of earlier blocks) is neither read nor written
template <typename Idx>
__device__ __forceinline__ void apply_fetch(ApplyRow &a, const ApplyMeta &m, const uint64_t *RX,
                                            const uint64_t *RZ, uint32_t rs, uint32_t word, uint32_t nrows,
                                            bool ok) {
  a.r = m.r;
  a.b = m.b;
  a.lo = m.lo;
  a.hi = m.hi;
  a.x = a.z = make_uint2(0, 0);
  if (ok && m.r < nrows) {
    const Idx off = (Idx)m.r * rs + word;
    a.x = reinterpret_cast<const uint2 *>(RX)[off];
    a.z = reinterpret_cast<const uint2 *>(RZ)[off];
  }
}

// a ^ b ^ c in one three-input logic operation
__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ void acc3(uint4 &a, const uint4 &p, const uint4 &q) {
  a.x = xor3(a.x, p.x, q.x);
  a.y = xor3(a.y, p.y, q.y);
  a.z = xor3(a.z, p.z, q.z);
  a.w = xor3(a.w, p.w, q.w);
}

constexpr int kSmemGroups = 8;            // shared-memory groups (steps 0..43)
constexpr int kSmemEntries = 7 * 64 + 4;  // 452 entries of 512 bytes
constexpr int kTmemStep0 = 44;            // first step held in TMEM
constexpr uint32_t kTmemCols = 512;       // all of the SM's tensor memory
__host__ __device__ constexpr int smem_group_bits(int g) { return g < 7 ? 6 : 2; }
__host__ __device__ constexpr int smem_group_base(int g) { return 64 * g; }

// byte offset (pattern * 512) of shared group g (6 steps from 6 g; group 7: steps 42, 43)
template <int g>
__device__ __forceinline__ uint32_t pat_off(uint32_t lo, uint32_t hi) {
  constexpr int sh = 6 * g, nb = smem_group_bits(g);
  constexpr uint32_t mask = (uint32_t)((1 << nb) - 1) * kEntryBytes;
  if constexpr (sh + nb <= 32) {
    if constexpr (sh >= 9) return (lo >> (sh - 9)) & mask;
    else return (lo << (9 - sh)) & mask;
  } else if constexpr (sh >= 32) {
    if constexpr (sh - 32 >= 9) return (hi >> (sh - 32 - 9)) & mask;
    else return (hi << (9 - (sh - 32))) & mask;
  } else {
    return __funnelshift_r(lo, hi, sh - 9) & mask;  // bits straddle the halves
  }
}

// shared table entry of group g for this lane: (x lo, x hi, z lo, z hi); the
// pattern's byte offset is a multiple of 512 and the lane's (16 lane) is
// below 512, so one OR joins them
template <int g>
__device__ __forceinline__ uint4 tab(const char *tb, uint32_t lane16, uint32_t lo, uint32_t hi) {
  return *reinterpret_cast<const uint4 *>(tb + smem_group_base(g) * kEntryBytes + (pat_off<g>(lo, hi) | lane16));
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint4 &v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(taddr));
}

// waits for this thread's TMEM loads; the operands tie the loaded registers
// to the wait so that no use is scheduled before it
__device__ __forceinline__ void tmem_wait_ld(uint4 &a, uint4 &b, uint4 &c, uint4 &d) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(a.x), "+r"(a.y), "+r"(a.z), "+r"(a.w), "+r"(b.x), "+r"(b.y), "+r"(b.z), "+r"(b.w),
                 "+r"(c.x), "+r"(c.y), "+r"(c.z), "+r"(c.w), "+r"(d.x), "+r"(d.y), "+r"(d.z), "+r"(d.w)
               :
               : "memory");
}

__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x),
               "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <typename Idx>
__device__ __forceinline__ void apply_row(const ApplyRow &a, uint32_t nrows, uint64_t *RX, uint64_t *RZ,
                                          bool ok, uint32_t word, const uint32_t *qubits,
                                          const uint64_t *VX, const uint64_t *VZ, uint32_t rs,
                                          uint32_t lane, const char *tb, uint32_t tq, int32_t *Tp,
                                          uint64_t tp0) {
  const uint32_t r = a.r;
  if (r >= nrows) return;  // uniform over the warp
  const Idx off = (Idx)r * rs + word;
  uint2 *px = reinterpret_cast<uint2 *>(RX), *pz = reinterpret_cast<uint2 *>(RZ);
  if (a.b >= kBasePivot) {  // pivot row of step j: +-Z_q (sign set by blk_rows_kernel)
    const uint32_t q = qubits[a.b - kBasePivot];
    if (ok) {
      px[off] = make_uint2(0, 0);
      const uint32_t bit = ((q >> 6) == word) ? 1u << (q & 31) : 0u;
      pz[off] = (q & 32) ? make_uint2(0, bit) : make_uint2(bit, 0);
    }
    return;
  }
  if (a.b == kBaseOrig && (a.lo | a.hi) == 0) return;
  uint2 xb = a.x, zb = a.z;
  if (a.b != kBaseOrig && ok) {  // destabilizer replaced by V_b at step b
    xb = reinterpret_cast<const uint2 *>(VX)[(uint64_t)a.b * rs + word];
    zb = reinterpret_cast<const uint2 *>(VZ)[(uint64_t)a.b * rs + word];
  }
  const uint32_t lo = a.lo, hi = a.hi;
  // steps 44..63 = bits 12..31 of hi: TMEM group t holds bits 12 + 5 t ..
  uint4 m0, m1, m2, m3;
  tmem_ld4(tq + 4 * ((hi >> 12) & 31), m0);
  tmem_ld4(tq + 128 + 4 * ((hi >> 17) & 31), m1);
  tmem_ld4(tq + 256 + 4 * ((hi >> 22) & 31), m2);
  tmem_ld4(tq + 384 + 4 * (hi >> 27), m3);
  const uint32_t l16 = lane * 16;
  uint4 acc = tab<0>(tb, l16, lo, hi);
  acc3(acc, tab<1>(tb, l16, lo, hi), tab<2>(tb, l16, lo, hi));
  acc3(acc, tab<3>(tb, l16, lo, hi), tab<4>(tb, l16, lo, hi));
  acc3(acc, tab<5>(tb, l16, lo, hi), tab<6>(tb, l16, lo, hi));
  const uint4 s7 = tab<7>(tb, l16, lo, hi);
  tmem_wait_ld(m0, m1, m2, m3);
  acc3(acc, s7, m0);
  acc3(acc, m1, m2);
  acc.x ^= m3.x;
  acc.y ^= m3.y;
  acc.z ^= m3.z;
  acc.w ^= m3.w;
  const uint2 xf = make_uint2(xb.x ^ acc.x, xb.y ^ acc.y), zf = make_uint2(zb.x ^ acc.z, zb.y ^ acc.w);
  if (ok) {
    px[off] = xf;
    pz[off] = zf;
  }
  const int t = __popc(xb.x & zb.x) + __popc(xb.y & zb.y) - __popc(xf.x & zf.x) - __popc(xf.y & zf.y);
  const int c = __popc((acc.z & xb.x) ^ (acc.w & xb.y)) & 1;  // parity of z_acc . x_b
  const int v = __reduce_add_sync(0xffffffffu, 64 * t + c);
  if (lane == 0) Tp[tp0 + r] = (v >> 6) * 2 + (v & 1);
}

// 1,024 threads at 64 registers: 6.80 ms per dense block at 180k, against
// 7.46 ms with 768 threads (80 registers) and 9.55 ms with 512 (100)
constexpr int kApplyThreads = 1024;
// blocks per SM over the grid: 6.41 ms per dense 180k block with 32 waves of
// one block per SM, 6.43 with 24, 6.49 with 16, 6.79 with 8, 7.46 with 4 (the
// tails of the last wave shrink; a block's table build stays small)
constexpr int kApplyWaves = 32;

template <typename Idx>
__global__ void __launch_bounds__(kApplyThreads, 1)
blk_apply_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint32_t rs, uint32_t nrows,
                 const uint32_t *__restrict__ window, const uint64_t *__restrict__ VX,
                 const uint64_t *__restrict__ VZ, const uint4 *__restrict__ list,
                 int32_t *__restrict__ Tp, const BlkState *st) {
  extern __shared__ ulonglong2 T[];  // [kSmemEntries][kCW] of (x word, z word)
  __shared__ uint32_t s_tmem;
  const int L = st->len;
  if (L == 0) return;  // a block enqueued past the window's end or behind a deterministic step
  const uint32_t *qubits = window + st->i0;
  const uint32_t u0 = blockIdx.x * kCW;  // first column word of the chunk
  const uint32_t nw = min((uint32_t)kCW, rs - u0);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {  // the whole TMEM of the SM: one block per SM (the tables fill shared memory)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // shared tables, one item per (group, quarter of its entries, word): the
  // quarter's two top steps give its first entry, then its entries follow in
  // Gray-code order, each one V row away from the previous
  for (int it = threadIdx.x; it < kSmemGroups * 4 * 32; it += blockDim.x) {
    const int w = it & 31, sr = (it >> 5) & 3, g = it >> 7;
    const int nb = smem_group_bits(g), e0 = smem_group_base(g) + (sr << (nb - 2));
    ulonglong2 vv[6];
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      const int st = 6 * g + b;
      vv[b] = make_ulonglong2(0, 0);
      if (b < nb && st < L && (uint32_t)w < nw)
        vv[b] = make_ulonglong2(VX[(uint64_t)st * rs + u0 + w], VZ[(uint64_t)st * rs + u0 + w]);
    }
    const ulonglong2 t0 = nb == 6 ? vv[4] : vv[0], t1 = nb == 6 ? vv[5] : vv[1];
    ulonglong2 e = make_ulonglong2(((sr & 1) ? t0.x : 0) ^ ((sr & 2) ? t1.x : 0),
                                   ((sr & 1) ? t0.y : 0) ^ ((sr & 2) ? t1.y : 0));
    T[e0 * kCW + w] = e;
    if (nb == 6) {
#pragma unroll
      for (int k = 1; k < 16; ++k) {
        const int lb = (k & 1) ? 0 : (k & 2) ? 1 : (k & 4) ? 2 : 3;
        e.x ^= vv[lb].x;
        e.y ^= vv[lb].y;
        T[(e0 + (k ^ (k >> 1))) * kCW + w] = e;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tq = s_tmem + ((32u * (warp & 3)) << 16);  // lane quarter of this warp
  if (warp < 16) {
    // TMEM table t = warp / 4 of this warp's quarter, entries in Gray-code order
    const int t = warp >> 2;
    uint4 v[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const int st = kTmemStep0 + 5 * t + b;
      v[b] = make_uint4(0, 0, 0, 0);
      if (st < L && lane < nw) {
        const uint2 x = reinterpret_cast<const uint2 *>(VX)[(uint64_t)st * rs + u0 + lane];
        const uint2 z = reinterpret_cast<const uint2 *>(VZ)[(uint64_t)st * rs + u0 + lane];
        v[b] = make_uint4(x.x, x.y, z.x, z.y);
      }
    }
    uint4 e = make_uint4(0, 0, 0, 0);
    tmem_st4(tq + 128 * t, e);
#pragma unroll
    for (int k = 1; k < 32; ++k) {
      const int b = (k & 1) ? 0 : (k & 2) ? 1 : (k & 4) ? 2 : (k & 8) ? 3 : 4;
      e.x ^= v[b].x;
      e.y ^= v[b].y;
      e.z ^= v[b].z;
      e.w ^= v[b].w;
      tmem_st4(tq + 128 * t + 4 * (k ^ (k >> 1)), e);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t cnt = st->ntouched;
  if (L > 0) {
    const bool ok = lane < nw;
    const uint32_t word = u0 + lane;
    const char *tb = reinterpret_cast<const char *>(T);
    const uint32_t units = gridDim.y * (blockDim.x >> 5);
    const uint64_t tp0 = (uint64_t)blockIdx.x * nrows;
    // the warp's entries of the row list: j, j + units, ...
    uint32_t j = blockIdx.y * (blockDim.x >> 5) + warp;
    ApplyRow a0, a1, a2;
    ApplyMeta mn;
    apply_meta(mn, j, cnt, nrows, list);
    apply_fetch<Idx>(a0, mn, RX, RZ, rs, word, nrows, ok);
    apply_meta(mn, j + units, cnt, nrows, list);
    apply_fetch<Idx>(a1, mn, RX, RZ, rs, word, nrows, ok);
    apply_meta(mn, j + 2 * units, cnt, nrows, list);
    for (; j < cnt; j += 3 * units) {
      apply_fetch<Idx>(a2, mn, RX, RZ, rs, word, nrows, ok);
      apply_meta(mn, j + 3 * units, cnt, nrows, list);
      apply_row<Idx>(a0, nrows, RX, RZ, ok, word, qubits, VX, VZ, rs, lane, tb, tq, Tp, tp0);
      apply_fetch<Idx>(a0, mn, RX, RZ, rs, word, nrows, ok);
      apply_meta(mn, j + 4 * units, cnt, nrows, list);
      apply_row<Idx>(a1, nrows, RX, RZ, ok, word, qubits, VX, VZ, rs, lane, tb, tq, Tp, tp0);
      apply_fetch<Idx>(a1, mn, RX, RZ, rs, word, nrows, ok);
      apply_meta(mn, j + 5 * units, cnt, nrows, list);
      apply_row<Idx>(a2, nrows, RX, RZ, ok, word, qubits, VX, VZ, rs, lane, tb, tq, Tp, tp0);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(kTmemCols)
                 : "memory");
  }
}

// per row: new sign from the accumulated terms; pivot rows get their coin; record
__global__ void __launch_bounds__(256)
blk_rows_kernel(uint64_t *__restrict__ S, uint64_t nrows, const uint64_t *__restrict__ M,
                const int32_t *__restrict__ base, const int32_t *__restrict__ Tp, uint32_t chunks,
                BlkState *st, uint64_t window_m0, uint64_t seed, uint64_t shot,
                uint8_t *__restrict__ record, uint8_t *__restrict__ kinds, uint32_t *__restrict__ err) {
  __shared__ int sw[64];          // 2 rV_s + A_s of each step
  __shared__ uint64_t sG[64];     // G rows
  const int L = st->len;
  const uint64_t m0 = window_m0 + st->i0;  // record index of the block's first measurement
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((int)threadIdx.x < L) {  // blockDim >= 64 >= L
    sw[threadIdx.x] = 2 * st->rV[threadIdx.x] + st->A[threadIdx.x];
    sG[threadIdx.x] = st->G[threadIdx.x];
  }
  __syncthreads();
  if (r == 0) st->cursor = st->i0 + (uint32_t)L;  // the next block starts here
  if (r < (uint64_t)L) {
    const uint32_t b = (uint32_t)(philox4x64_10(m0 + r, shot, 0, 0, seed, kCoinKey).v[0] & 1u);
    record[m0 + r] = (uint8_t)b;
    kinds[m0 + r] = 1;  // every step of a block had a pivot
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
        e += sw[s];
      }
      e += 2 * cross_pairs(sG, sr);
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
         2 * al(64ull * L.rs * 8) + al(sizeof(BlkState)) + al(L.nrows * 16);
}

static std::atomic<uint64_t> g_apply_attr_set{0};

// Enqueues one block of up to 64 measurements; the number actually done is
// st->len (read by the host after the stream is synchronised).
cudaError_t launch_measure_block(const Dev &d, void *scratch, const uint32_t *window, uint32_t count,
                                 uint64_t m0, qs_key key, cudaStream_t s, int *launches) {
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
  uint4 *list = reinterpret_cast<uint4 *>(take(L.nrows * 16));
  const unsigned rb = (unsigned)((L.nrows + 255) / 256);
  const size_t smem = (size_t)kSmemEntries * kEntryBytes;
  cudaError_t ea = once_per_device(g_apply_attr_set, [&]() {
    cudaError_t e = cudaFuncSetAttribute(blk_apply_kernel<uint32_t>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(blk_apply_kernel<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(blk_vrows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kVrowSmem);
    return e;
  });
  if (ea != cudaSuccess) return ea;
  tbegin(d.timer, QS_TIME_BLK_SYMBOLIC, s);
  const uint32_t nwin = (L.n + kLazyThreads - 1) >> kLazyLog2;
  blk_reset_kernel<<<1, 256, 0, s>>>(st, count, nwin);
  blk_init_kernel<<<rb, 256, 0, s>>>(d.RX, L.rs, L.nrows, L.n, L.k, window, C0, M, base, st, d.err);
  int sym_launches = 64;
  if (!d.step_symbolic) {
    blk_lazy_symbolic_kernel<<<1, kLazyThreads, 0, s>>>(L.n, L.k, C0, C1, st);
    blk_replay_kernel<<<rb, 256, 0, s>>>(L.nrows, L.k, C0, M, base, st);
    sym_launches = 2;
  } else {
    for (int j = 0; j < 64; ++j)  // steps past the block's length return at once
      blk_step_kernel<<<rb, 256, 0, s>>>(L.nrows, L.n, L.k, j, (j & 1) ? C1 : C0, (j & 1) ? C0 : C1, M,
                                         base, st);
  }
  tend(d.timer, QS_TIME_BLK_SYMBOLIC, s);
  tbegin(d.timer, QS_TIME_BLK_PIVOT_ROWS, s);
  blk_vrows_kernel<<<dim3(chunks, kVrowSplit), kVrowThreads, kVrowSmem, s>>>(d.RX, d.RZ, L.rs, VX,
                                                                              VZ, st);
  blk_signs_kernel<<<1, 64, 0, s>>>(d.S, st, d.err);
  blk_list_kernel<<<rb, 256, 0, s>>>(L.nrows, M, base, list, st);
  tend(d.timer, QS_TIME_BLK_PIVOT_ROWS, s);
  // about kApplyWaves waves of one block per SM (the tables take 226 KB of
  // shared memory and all of TMEM), but at least 512 rows per block so that
  // building the tables stays small next to the rows they serve
  const uint32_t rows_y = std::max<uint32_t>(
      1, (uint32_t)std::min<uint64_t>(((uint64_t)d.sms * kApplyWaves + chunks - 1) / chunks, L.nrows / 512));
  tbegin(d.timer, QS_TIME_BLK_APPLY, s);
  if (!d.wide_offsets && (uint64_t)L.nrows * L.rs < (1ull << 32))
    blk_apply_kernel<uint32_t><<<dim3(chunks, rows_y), kApplyThreads, smem, s>>>(
        d.RX, d.RZ, L.rs, (uint32_t)L.nrows, window, VX, VZ, list, Tp, st);
  else
    blk_apply_kernel<uint64_t><<<dim3(chunks, rows_y), kApplyThreads, smem, s>>>(
        d.RX, d.RZ, L.rs, (uint32_t)L.nrows, window, VX, VZ, list, Tp, st);
  tend(d.timer, QS_TIME_BLK_APPLY, s);
  tbegin(d.timer, QS_TIME_BLK_SIGNS, s);
  blk_rows_kernel<<<rb, 256, 0, s>>>(d.S, L.nrows, M, base, Tp, chunks, st, m0, key.seed, key.shot,
                                     d.record, d.kinds, d.err);
  tend(d.timer, QS_TIME_BLK_SIGNS, s);
  if (launches) *launches += 7 + sym_launches;
  return cudaGetLastError();
}

__global__ void blk_set_cursor_kernel(BlkState *st, uint32_t v) { st->cursor = v; }

static BlkState *blk_state(const Layout &L, void *scratch) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  return reinterpret_cast<BlkState *>(static_cast<uint8_t *>(scratch) + 3 * al(L.nrows * 8) +
                                      al(L.nrows * 4) + al((size_t)blk_chunks(L) * L.nrows * 4) +
                                      2 * al(64ull * L.rs * 8));
}

cudaError_t set_block_cursor(const Layout &L, void *scratch, uint32_t v, cudaStream_t s) {
  blk_set_cursor_kernel<<<1, 1, 0, s>>>(blk_state(L, scratch), v);
  return cudaGetLastError();
}

const uint32_t *block_cursor(const Layout &L, void *scratch) { return &blk_state(L, scratch)->cursor; }


}  // namespace qs
