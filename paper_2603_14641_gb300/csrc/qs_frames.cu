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

}  // namespace qs
