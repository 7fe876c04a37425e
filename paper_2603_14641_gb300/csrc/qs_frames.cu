// Pauli-frame many-shot sampling, Sec. 5 (Alg. 9).
//
// Frames are two bit matrices X~, Z~ stored per qubit as fw 64-bit shot words
// (bit s of word j = shot 64 j + s), the layout of Alg. 9 with one word
// holding 64 shots of one qubit. Gate layers reuse the column-major gate
// kernel with signs compiled out (qs_gates.cu).
//   Randomize (Alg. 9 init):  X~ = 0; Z~[q][j] = word (j & 3) of
//                             Philox(ctr = (0, q, j >> 2, 1), key = (seed, 0xF4A3E)).
//   MeasureSample (Alg. 9):   out[m][j] = X~[q][j] XOR (ref[m] ? ~0 : 0),
//                             Z~[q][j] = word (j & 3) of Philox(ctr = (m + 1, q, j >> 2, 1), ...).
// The XOR with the reference record is the reading of Alg. 9 that makes the
// output a sample (the frames carry flips relative to one valid record).
//   Noise (frames carry error events, Sec. 3): target i of noise op e fires
//                             in shot s iff u < floor(p 2^32); bit 31 - k of u
//                             is bit (s & 63) of word (k & 3) of
//                             Philox(ctr = (e, i, 8 (s >> 6) + (k >> 2), 3),
//                             key = (seed, 0xE5505));
//                             the Pauli of a depolarising channel comes from
//                             word 0 of Philox(ctr = (e, i, s, 4), same key).
#include "qs_internal.cuh"

namespace qs {

// fw is a multiple of 4: one Philox block fills 4 consecutive shot words
__global__ void frame_init_kernel(uint64_t *__restrict__ FZ, uint32_t n, uint32_t fw, uint64_t seed) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t quads = fw >> 2;
  const uint64_t total = (uint64_t)n * quads;
  if (idx >= total) return;
  const uint32_t q = (uint32_t)(idx / quads), j4 = (uint32_t)(idx % quads);
  P4 r = philox4x64_10(0, q, j4, 1, seed, kFrameKey);
  ulonglong2 *p = reinterpret_cast<ulonglong2 *>(FZ + (uint64_t)q * fw + 4ull * j4);
  p[0] = make_ulonglong2(r.v[0], r.v[1]);
  p[1] = make_ulonglong2(r.v[2], r.v[3]);
}

cudaError_t launch_frame_init(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw, uint64_t seed,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(FX, 0, (size_t)n * fw * sizeof(uint64_t), s);
  if (e != cudaSuccess) return e;
  const uint64_t total = (uint64_t)n * (fw >> 2);
  frame_init_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(FZ, n, fw, seed);
  return cudaGetLastError();
}

// grid.x over shot-word quads, grid.y over the measurements of the window
// (the qubits of one launch are distinct)
__global__ void frame_measure_kernel(const uint64_t *__restrict__ FX, uint64_t *__restrict__ FZ,
                                     uint32_t n, uint32_t fw, const uint32_t *__restrict__ qubits,
                                     uint64_t m0, const uint8_t *__restrict__ ref,
                                     uint64_t *__restrict__ out, uint64_t shots, uint64_t seed,
                                     uint32_t *__restrict__ err) {
  const uint32_t i = blockIdx.y;
  const uint32_t j4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (j4 >= (fw >> 2)) return;
  const uint32_t q = qubits[i];
  if (q >= n) {
    if (j4 == 0) atomicOr(err, kErrBadQubit);
    return;
  }
  const uint64_t m = m0 + i;
  const uint64_t ow = (shots + 63) / 64;  // output words per measurement
  const uint64_t flip = ref[m] ? ~0ull : 0ull;
  const uint64_t *fx = FX + (uint64_t)q * fw + 4ull * j4;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const uint64_t j = 4ull * j4 + t;
    if (j < ow) {
      uint64_t v = fx[t] ^ flip;
      if (j == ow - 1 && (shots & 63)) v &= (1ull << (shots & 63)) - 1;
      out[m * ow + j] = v;
    }
  }
  P4 r = philox4x64_10(m + 1, q, j4, 1, seed, kFrameKey);
  ulonglong2 *pz = reinterpret_cast<ulonglong2 *>(FZ + (uint64_t)q * fw + 4ull * j4);
  pz[0] = make_ulonglong2(r.v[0], r.v[1]);
  pz[1] = make_ulonglong2(r.v[2], r.v[3]);
}

cudaError_t launch_frame_measure(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw,
                                 const uint32_t *qubits, uint32_t count, uint64_t m0,
                                 const uint8_t *ref, uint64_t *out, uint64_t shots, uint64_t seed,
                                 uint32_t *err, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const uint32_t quads = fw >> 2;
  const uint32_t threads = quads < 128 ? ((quads + 31) / 32) * 32 : 128;
  // grid.y is limited to 65535: split long windows
  for (uint32_t off = 0; off < count; off += 65535) {
    const uint32_t c = count - off < 65535 ? count - off : 65535;
    dim3 grid((quads + threads - 1) / threads, c);
    frame_measure_kernel<<<grid, threads, 0, s>>>(FX, FZ, n, fw, qubits + off, m0 + off, ref, out,
                                                  shots, seed, err);
  }
  return cudaGetLastError();
}

// Pauli noise channels on the frames (X_ERROR, Y_ERROR, Z_ERROR, DEPOLARIZE1,
// DEPOLARIZE2; frames carry error events, Sec. 3). One thread per (target,
// shot word j). The 64 shots' 32-bit draws u are bit-sliced: bit 31 - k of
// every shot's u sits in random word W_k, so u < thr is decided for all 64
// shots at once from the most significant bit down, and the loop stops as
// soon as no shot is undecided (about 8 words on average instead of 32).
// The fire mask applies X/Y/Z directly; only the shots that fired draw the
// Pauli of a depolarising channel. Targets of one op are distinct, so every
// frame word has one writer.
__device__ __forceinline__ uint64_t noise_v(uint64_t e, uint64_t i, uint64_t s, uint64_t seed) {
  return philox4x64_10(e, i, s, 4, seed, kNoiseKey).v[0];
}
__device__ __forceinline__ void add_pauli(int code, uint64_t bit, uint64_t &mx, uint64_t &mz) {
  if (code == 1 || code == 2) mx |= bit;
  if (code == 2 || code == 3) mz |= bit;
}

__global__ void __launch_bounds__(256)
frame_noise_kernel(uint64_t *__restrict__ FX, uint64_t *__restrict__ FZ, uint32_t fw, uint32_t ow,
                   const uint32_t *__restrict__ targets, uint32_t count, uint32_t i0, int kind,
                   uint64_t thr, uint64_t e, uint64_t seed) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (uint64_t)count * ow) return;
  const uint32_t i = (uint32_t)(tid / ow), j = (uint32_t)(tid % ow);
  const uint64_t gi = (uint64_t)i0 + i;
  uint64_t fire = 0;
  if (thr >> 32) {
    fire = ~0ull;  // p >= 1
  } else {
    uint64_t undecided = ~0ull;
    for (int t = 0; t < 8 && undecided; ++t) {
      const P4 r = philox4x64_10(e, gi, 8ull * j + t, 3, seed, kNoiseKey);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint64_t w = r.v[q];  // bit 31 - (4 t + q) of every shot's u
        if ((thr >> (31 - (4 * t + q))) & 1u) {
          fire |= undecided & ~w;  // u has 0 where thr has 1: u < thr
          undecided &= w;
        } else {
          undecided &= ~w;  // u has 1 where thr has 0: u > thr
        }
      }
    }
    // shots still undecided after 32 bits have u == thr: no fire
  }
  if (!fire) return;
  uint64_t ax = 0, az = 0, bx = 0, bz = 0;
  if (kind == QS_NOISE_X) ax = fire;
  else if (kind == QS_NOISE_Y) ax = az = fire;
  else if (kind == QS_NOISE_Z) az = fire;
  else {
    uint64_t m = fire;
    while (m) {
      const int b = __ffsll((long long)m) - 1;
      m &= m - 1;
      const uint64_t v = noise_v(e, gi, 64ull * j + b, seed), bit = 1ull << b;
      if (kind == QS_NOISE_DEPOLARIZE1) {
        add_pauli(1 + (int)__umul64hi(v, 3), bit, ax, az);
      } else {
        const int idx = 1 + (int)__umul64hi(v, 15);
        add_pauli(idx >> 2, bit, ax, az);
        add_pauli(idx & 3, bit, bx, bz);
      }
    }
  }
  const uint64_t qa = kind == QS_NOISE_DEPOLARIZE2 ? targets[2 * i] : targets[i];
  if (ax) FX[qa * fw + j] ^= ax;
  if (az) FZ[qa * fw + j] ^= az;
  if (kind == QS_NOISE_DEPOLARIZE2) {
    const uint64_t qb = targets[2 * i + 1];
    if (bx) FX[qb * fw + j] ^= bx;
    if (bz) FZ[qb * fw + j] ^= bz;
  }
}

cudaError_t launch_frame_noise(uint64_t *FX, uint64_t *FZ, uint32_t fw, uint32_t ow,
                               const uint32_t *targets, uint32_t count, uint32_t i0, int kind,
                               uint64_t thr, uint64_t e, uint64_t seed, cudaStream_t s) {
  if (count == 0 || ow == 0 || thr == 0) return cudaSuccess;  // never fires
  const uint64_t threads = (uint64_t)count * ow;
  const uint64_t blocks = (threads + 255) / 256;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  frame_noise_kernel<<<(unsigned)blocks, 256, 0, s>>>(FX, FZ, fw, ow, targets, count, i0, kind, thr,
                                                      e, seed);
  return cudaGetLastError();
}

}  // namespace qs
