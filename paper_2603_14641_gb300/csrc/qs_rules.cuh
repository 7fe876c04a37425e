// Per-word Clifford update rules shared by the fused and batched kernels.
//
// Sec. 2.4 Eq. 4 gives H, P and CX; the rest of the paper's 11-gate set
// (Sec. 6) is the composition of those rules evaluated in registers:
// S^dag = S^3, CZ = H_t CX H_t, CY = S_t CX S_t^dag (circuit order S_t^dag,
// CX, S_t), SWAP, ISWAP = CZ, SWAP, S_a, S_b (circuit order). Each call updates
// one 64-bit word (64 rows) of the columns of qubits a (and b) and XORs the
// sign contribution into s. With SIGNS = false (Pauli frames) X/Y/Z change
// nothing and S^dag acts like S.
#pragma once

#include <stdint.h>

#include "../../include/qs.h"

namespace qs {

template <bool SIGNS>
__device__ __forceinline__ void rule(uint32_t type, uint64_t &xa, uint64_t &za, uint64_t &xb,
                                     uint64_t &zb, uint64_t &s) {
  switch (type) {
    case QS_X: if (SIGNS) s ^= za; break;
    case QS_Z: if (SIGNS) s ^= xa; break;
    case QS_Y: if (SIGNS) s ^= xa ^ za; break;
    case QS_H: { if (SIGNS) s ^= xa & za; uint64_t t = xa; xa = za; za = t; } break;
    case QS_S: if (SIGNS) s ^= xa & za; za ^= xa; break;
    case QS_SDG: if (SIGNS) s ^= xa & ~za; za ^= xa; break;
    case QS_CX:
      if (SIGNS) s ^= xa & zb & ~(xb ^ za);
      xb ^= xa; za ^= zb; break;
    case QS_CZ:
      if (SIGNS) s ^= xa & xb & (za ^ zb);
      za ^= xb; zb ^= xa; break;
    case QS_CY:  // S_b^dag, CX(a, b), S_b
      if (SIGNS) s ^= xb & ~zb;
      zb ^= xb;
      if (SIGNS) s ^= xa & zb & ~(xb ^ za);
      xb ^= xa; za ^= zb;
      if (SIGNS) s ^= xb & zb;
      zb ^= xb; break;
    case QS_SWAP: { uint64_t t = xa; xa = xb; xb = t; t = za; za = zb; zb = t; } break;
    case QS_ISWAP: {  // CZ, SWAP, S_a, S_b
      if (SIGNS) s ^= xa & xb & (za ^ zb);
      uint64_t nza = za ^ xb, nzb = zb ^ xa;
      uint64_t t = xa; xa = xb; xb = t;
      za = nzb; zb = nza;
      if (SIGNS) s ^= xa & za;
      za ^= xa;
      if (SIGNS) s ^= xb & zb;
      zb ^= xb;
    } break;
    default: break;
  }
}

}  // namespace qs
