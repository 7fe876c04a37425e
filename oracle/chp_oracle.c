/*
 * CPU oracle: a plain, single-threaded CHP stabilizer simulator over unpacked
 * bit rows (one uint8_t per tableau bit).
 *
 * TEST INFRASTRUCTURE ONLY. It exists to check the CUDA path; only tests, the
 * smoke check and the benchmark's CPU-baseline leg load it. It shares no code,
 * header or table with the CUDA library, and it is written for clarity, not
 * speed.
 *
 * What it computes (paper: arXiv 2603.14641):
 *   - Extended tableau of Sec. 2.5, Eq. 7: rows 0..n-1 are destabilizers
 *     D_1..D_n, rows n..2n-1 stabilizers S_1..S_n; each row holds x bits,
 *     z bits and a sign bit r (generator = (-1)^r * P, P encoded per qubit
 *     by (x,z): (0,0)=I, (1,0)=X, (1,1)=Y, (0,1)=Z, Sec. 2.4).
 *   - Gates H, P(=S), CX by the column update rules of Sec. 2.4, Eq. 4,
 *     applied to every row. The rest of the 11-gate set of Sec. 6 is built
 *     from those rules (X/Y/Z flip the sign of anticommuting rows; S^dag =
 *     S^3; CZ = H_t CX H_t; CY = S_t CX S_t^dag; SWAP = 3 CX;
 *     ISWAP = CZ, SWAP, S_a, S_b in circuit order).
 *   - Z-measurement by the CHP algorithm of Sec. 2.5: pivot = smallest
 *     stabilizer with x_pq = 1; rowsum of the pivot into every other row
 *     with x_iq = 1; D_p <- S_p; S_p <- (-1)^m Z_q with m a fresh coin; in the
 *     deterministic case (-1)^m Z_q = product of S_i over destabilizers D_i
 *     that anticommute with Z_q, accumulated in a scratch row.
 *   - rowsum(h, i) of Aaronson & Gottesman (cited in Sec. 2.5): the phase is
 *     2 r_h + 2 r_i + sum_j g(x_ij, z_ij, x_hj, z_hj) mod 4, where g is the
 *     exponent of i in the single-qubit product sigma(x_ij,z_ij) *
 *     sigma(x_hj,z_hj).
 *   - The paper's measurement variant (Sec. 3.2, Alg. 1: Stim's elimination by
 *     CX injection) on the inverse tableau with qubit-indexed signs, with its
 *     own gate rules for those signs (the oracle_inv_* functions below).
 *   - Pauli-frame sampling of Sec. 5 (Alg. 9) with a reference record
 *     (the frames carry flips relative to that record).
 *   - Pauli noise channels on the frames (Sec. 3 notes that frames carry
 *     error events as well as measurement randomness; the paper fixes no
 *     channel set or sampling rule, so these are a reading): X_ERROR(p),
 *     Y_ERROR(p), Z_ERROR(p) apply their Pauli with probability p;
 *     DEPOLARIZE1(p) applies one of X, Y, Z, each with probability p/3;
 *     DEPOLARIZE2(p) applies one of the 15 non-identity two-qubit Paulis,
 *     each with probability p/15. The tableau (reference shot) is noiseless.
 *
 * Readings of the paper where it is silent or garbled (listed in the design
 * notes): the rowsum goes into every row i != p (both halves) with x_iq = 1,
 * skipping the paired destabilizer p-n that is overwritten right after;
 * destabilizer signs follow the same update rules; the coin is a keyed
 * Philox4x64-10 bit.
 *
 * Keyed randomness: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 * written here from its published definition:
 *   coin(seed, shot, m)      = bit 0 of word 0 of Philox(ctr=(m, shot, 0, 0),
 *                                                     key=(seed, 0x51A7E))
 *   frame_word(seed, e, q, j) = word (j & 3) of Philox(ctr=(e, q, j >> 2, 1),
 *                                                     key=(seed, 0xF4A3E))
 *   noise_u(seed, e, i, s)  = the 32-bit number whose bit 31 - k is bit
 *       (s & 63) of W_k, k = 0..31, W_k = word (k & 3) of
 *       Philox(ctr=(e, i, 8 (s >> 6) + (k >> 2), 3), key=(seed, 0xE5505))
 *   noise_v(seed, e, i, s)  = word 0 of Philox(ctr=(e, i, s, 4),
 *                                              key=(seed, 0xE5505))
 *       for target i of noise op e (ops numbered from 0 in program order)
 *       and shot s. The channel fires iff p >= 1 or u < floor(p * 2^32);
 *       when it fires, the Pauli is 1 + floor(3 v / 2^64) (1 = X, 2 = Y,
 *       3 = Z) for DEPOLARIZE1, or the two-qubit Pauli with index
 *       1 + floor(15 v / 2^64) = 4 a + b (0 = I, 1 = X, 2 = Y, 3 = Z).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon et al. 2011)                                   */
/* ------------------------------------------------------------------ */

static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  /* 64x64 -> 128 product from four 32x32 partial products */
  uint64_t a0 = a & 0xffffffffu, a1 = a >> 32, b0 = b & 0xffffffffu, b1 = b >> 32;
  uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
  uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
  *lo = (mid << 32) | (p00 & 0xffffffffu);
  *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void oracle_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t hi0, lo0, hi1, lo1;
    mul128(0xD2E7470EE14C6C93ull, c0, &hi0, &lo0);
    mul128(0xCA5A826395121157ull, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B97F4A7C15ull; /* Weyl key schedule */
    k1 += 0xBB67AE8584CAA73Bull;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

int oracle_coin(uint64_t seed, uint64_t shot, uint64_t m) {
  uint64_t ctr[4] = {m, shot, 0, 0}, key[2] = {seed, 0x51A7Eull}, out[4];
  oracle_philox4x64_10(ctr, key, out);
  return (int)(out[0] & 1u);
}

uint64_t oracle_frame_word(uint64_t seed, uint64_t e, uint64_t q, uint64_t j) {
  uint64_t ctr[4] = {e, q, j >> 2, 1}, key[2] = {seed, 0xF4A3Eull}, out[4];
  oracle_philox4x64_10(ctr, key, out);
  return out[j & 3];
}

void oracle_noise_draw(uint64_t seed, uint64_t e, uint64_t i, uint64_t s, uint64_t *u, uint64_t *v) {
  uint64_t key[2] = {seed, 0xE5505ull}, out[4];
  uint64_t j = s >> 6, b = s & 63u, acc = 0;
  for (int t = 0; t < 8; ++t) { /* block t holds W_{4t} .. W_{4t+3} */
    uint64_t cu[4] = {e, i, 8u * j + (uint64_t)t, 3};
    oracle_philox4x64_10(cu, key, out);
    for (int q = 0; q < 4; ++q) acc |= ((out[q] >> b) & 1u) << (31 - (4 * t + q));
  }
  *u = acc;
  uint64_t cv[4] = {e, i, s, 4};
  oracle_philox4x64_10(cv, key, out);
  *v = out[0];
}

/* floor(p * 2^32) for 0 <= p < 1 (multiplying by a power of two is exact);
 * 0 for p <= 0 and 2^32 for p >= 1 */
uint64_t oracle_noise_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return 4294967296ull;
  return (uint64_t)(p * 4294967296.0);
}

/* floor(v * k / 2^64): the high word of the 128-bit product */
static uint64_t mul_hi(uint64_t v, uint64_t k) {
  uint64_t hi, lo;
  mul128(v, k, &hi, &lo);
  return hi;
}

/* ------------------------------------------------------------------ */
/* Tableau                                                              */
/* ------------------------------------------------------------------ */

enum { G_I, G_X, G_Y, G_Z, G_H, G_S, G_SDG, G_CX, G_CY, G_CZ, G_SWAP, G_ISWAP };

typedef struct {
  int n;
  int rows;   /* rows the gate rules act on: 2n, or the size of a row subset */
  uint8_t *x; /* (2n+1) rows of n bits; row 2n is the scratch row */
  uint8_t *z;
  uint8_t *r; /* 2n+1 sign bits */
  long odd_phase_count; /* rowsums whose phase was odd (must stay 0) */
  long det_check_fail;  /* deterministic products that were not +-Z_q */
  int last_kind;        /* 1 = last measurement was probabilistic, 0 = deterministic */
} chp_t;

#define XB(t, i, j) ((t)->x[(size_t)(i) * (size_t)(t)->n + (size_t)(j)])
#define ZB(t, i, j) ((t)->z[(size_t)(i) * (size_t)(t)->n + (size_t)(j)])

void oracle_reset(chp_t *t, const uint8_t *initstate) {
  int n = t->n;
  memset(t->x, 0, (size_t)(2 * n + 1) * n);
  memset(t->z, 0, (size_t)(2 * n + 1) * n);
  memset(t->r, 0, (size_t)(2 * n + 1));
  for (int i = 0; i < n; ++i) {
    XB(t, i, i) = 1;      /* D_i = X_i */
    ZB(t, n + i, i) = 1;  /* S_i = Z_i */
    if (initstate && initstate[i]) { t->r[i] = 1; t->r[n + i] = 1; }
  }
  t->odd_phase_count = 0;
  t->det_check_fail = 0;
  t->last_kind = -1;
}

static void fill_g_table(void);

chp_t *oracle_new(int n) {
  fill_g_table(); /* the rowsum's g lookup (same values on every call) */
  chp_t *t = (chp_t *)calloc(1, sizeof(chp_t));
  if (!t) return NULL;
  t->n = n;
  t->rows = 2 * n;
  size_t cells = (size_t)(2 * n + 1) * (size_t)(n > 0 ? n : 1);
  t->x = (uint8_t *)calloc(cells, 1);
  t->z = (uint8_t *)calloc(cells, 1);
  t->r = (uint8_t *)calloc((size_t)(2 * n + 1), 1);
  if (!t->x || !t->z || !t->r) { free(t->x); free(t->z); free(t->r); free(t); return NULL; }
  oracle_reset(t, NULL);
  return t;
}

/* A subset of generator rows evolved under gates only. Gate rules act on
 * each row independently (Sec. 2.4: the rules apply to every row index i), so
 * rows row_ids[0..nr) (0..n-1 destabilizers, n..2n-1 stabilizers) of the
 * full tableau can be followed alone; row j of this object is row row_ids[j]
 * of the initial tableau |0...0>. */
chp_t *oracle_new_subset(int n, const uint32_t *row_ids, int nr) {
  chp_t *t = (chp_t *)calloc(1, sizeof(chp_t));
  if (!t) return NULL;
  t->n = n;
  t->rows = nr;
  size_t cells = (size_t)(nr + 1) * (size_t)n;
  t->x = (uint8_t *)calloc(cells, 1);
  t->z = (uint8_t *)calloc(cells, 1);
  t->r = (uint8_t *)calloc((size_t)nr + 1, 1);
  if (!t->x || !t->z || !t->r) { free(t->x); free(t->z); free(t->r); free(t); return NULL; }
  for (int j = 0; j < nr; ++j) {
    uint32_t g = row_ids[j];
    if (g < (uint32_t)n) XB(t, j, g) = 1;
    else ZB(t, j, g - (uint32_t)n) = 1;
  }
  t->last_kind = -1;
  return t;
}

/* Copies out the rows of a subset object: x, z are nr*n bytes, r is nr bytes. */
void oracle_get_subset(const chp_t *t, uint8_t *x, uint8_t *z, uint8_t *r) {
  size_t cells = (size_t)t->rows * t->n;
  memcpy(x, t->x, cells); memcpy(z, t->z, cells); memcpy(r, t->r, (size_t)t->rows);
}

void oracle_free(chp_t *t) {
  if (!t) return;
  free(t->x); free(t->z); free(t->r); free(t);
}

int oracle_n(const chp_t *t) { return t->n; }
long oracle_odd_phase_count(const chp_t *t) { return t->odd_phase_count; }
long oracle_det_check_fail(const chp_t *t) { return t->det_check_fail; }
int oracle_last_kind(const chp_t *t) { return t->last_kind; }

/* Copy out / in the 2n rows: x, z are 2n*n bytes (row-major), r is 2n bytes. */
void oracle_get(const chp_t *t, uint8_t *x, uint8_t *z, uint8_t *r) {
  size_t cells = (size_t)(2 * t->n) * t->n;
  memcpy(x, t->x, cells); memcpy(z, t->z, cells); memcpy(r, t->r, (size_t)(2 * t->n));
}
void oracle_set(chp_t *t, const uint8_t *x, const uint8_t *z, const uint8_t *r) {
  size_t cells = (size_t)(2 * t->n) * t->n;
  memcpy(t->x, x, cells); memcpy(t->z, z, cells); memcpy(t->r, r, (size_t)(2 * t->n));
}

/* --- Sec. 2.4, Eq. 4: the three base rules, on one row i --------------- */
/* Eq. 4 applies each rule to every row index i, and a row's new bits and sign
 * depend on that row alone, so the rules are written for one row and the
 * callers below run them over the rows. */

static void rule_h(chp_t *t, int i, int q) {
  uint8_t x = XB(t, i, q), z = ZB(t, i, q);
  t->r[i] ^= (uint8_t)(x & z);
  XB(t, i, q) = z;
  ZB(t, i, q) = x;
}

static void rule_p(chp_t *t, int i, int q) {
  uint8_t x = XB(t, i, q), z = ZB(t, i, q);
  t->r[i] ^= (uint8_t)(x & z);
  ZB(t, i, q) = (uint8_t)(z ^ x);
}

static void rule_cx(chp_t *t, int i, int c, int tq) {
  uint8_t xc = XB(t, i, c), zc = ZB(t, i, c), xt = XB(t, i, tq), zt = ZB(t, i, tq);
  t->r[i] ^= (uint8_t)(xc & zt & ((xt ^ zc) ^ 1u));
  XB(t, i, tq) = (uint8_t)(xt ^ xc);
  ZB(t, i, c) = (uint8_t)(zc ^ zt);
}

/* Pauli gates: conjugation by a Pauli flips the sign of exactly the rows
 * that anticommute with it on that qubit. */
static void rule_pauli(chp_t *t, int i, int q, int ax, int az) {
  /* the gate Pauli is (ax, az); a row Pauli (x, z) anticommutes with it
   * iff x*az + z*ax is odd */
  t->r[i] ^= (uint8_t)((XB(t, i, q) & az) ^ (ZB(t, i, q) & ax));
}

/* One gate on row i. */
static void gate_row(chp_t *t, int i, int type, int a, int b) {
  switch (type) {
    case G_I: break;
    case G_X: rule_pauli(t, i, a, 1, 0); break;
    case G_Y: rule_pauli(t, i, a, 1, 1); break;
    case G_Z: rule_pauli(t, i, a, 0, 1); break;
    case G_H: rule_h(t, i, a); break;
    case G_S: rule_p(t, i, a); break;
    case G_SDG: rule_p(t, i, a); rule_p(t, i, a); rule_p(t, i, a); break;
    case G_CX: rule_cx(t, i, a, b); break;
    case G_CZ: rule_h(t, i, b); rule_cx(t, i, a, b); rule_h(t, i, b); break;
    case G_CY: /* S_b^dag, CX, S_b in circuit order */
      rule_p(t, i, b); rule_p(t, i, b); rule_p(t, i, b); rule_cx(t, i, a, b); rule_p(t, i, b); break;
    case G_SWAP: rule_cx(t, i, a, b); rule_cx(t, i, b, a); rule_cx(t, i, a, b); break;
    case G_ISWAP: /* CZ, SWAP, S_a, S_b in circuit order */
      gate_row(t, i, G_CZ, a, b); gate_row(t, i, G_SWAP, a, b); rule_p(t, i, a); rule_p(t, i, b); break;
    default: break;
  }
}

void oracle_gate(chp_t *t, int type, int a, int b) {
  for (int i = 0; i < t->rows; ++i) gate_row(t, i, type, a, b);
}

/* gates: count rows of (type, q0, q1), applied in order. Every row goes
 * through the whole list before the next row starts: rows evolve
 * independently (Eq. 4 acts on each row index on its own), so this gives the
 * same tableau as applying gate by gate to all rows, while each row's bytes
 * stay in cache. */
void oracle_apply(chp_t *t, const uint32_t *gates, long count) {
  for (int i = 0; i < t->rows; ++i)
    for (long g = 0; g < count; ++g)
      gate_row(t, i, (int)gates[3 * g], (int)gates[3 * g + 1], (int)gates[3 * g + 2]);
}

/* --- rowsum (Aaronson & Gottesman), cited in Sec. 2.5 ------------------ */

/* exponent of i in sigma(x1,z1) * sigma(x2,z2), in {-1, 0, +1} */
static int g_fn(int x1, int z1, int x2, int z2) {
  if (x1 == 0 && z1 == 0) return 0;
  if (x1 == 1 && z1 == 1) return z2 - x2;           /* Y * . */
  if (x1 == 1 && z1 == 0) return z2 * (2 * x2 - 1); /* X * . */
  return x2 * (1 - 2 * z2);                         /* Z * . */
}

/* g_fn tabulated over its 16 arguments, index 8 x1 + 4 z1 + 2 x2 + z2 (a
 * lookup instead of branches on random bits; filled from g_fn itself) */
static int g_table[16];

static void fill_g_table(void) {
  for (int v = 0; v < 16; ++v) g_table[v] = g_fn((v >> 3) & 1, (v >> 2) & 1, (v >> 1) & 1, v & 1);
}

/* row h <- row i * row h (generator product), sign from the mod-4 phase */
static void rowsum(chp_t *t, int h, int i) {
  int n = t->n;
  long sum = 2 * (long)t->r[h] + 2 * (long)t->r[i];
  for (int j = 0; j < n; ++j)
    sum += g_table[8 * XB(t, i, j) + 4 * ZB(t, i, j) + 2 * XB(t, h, j) + ZB(t, h, j)];
  long m = ((sum % 4) + 4) % 4;
  if (m == 1 || m == 3) t->odd_phase_count++;
  t->r[h] = (uint8_t)(m == 2);
  for (int j = 0; j < n; ++j) {
    XB(t, h, j) ^= XB(t, i, j);
    ZB(t, h, j) ^= ZB(t, i, j);
  }
}

/* --- Z-measurement, Sec. 2.5 "The CHP algorithm" ---------------------- */

/* Measures qubit q. The coin of a probabilistic outcome is
 * coin(seed, shot, midx), or 0 when force_zero is set (reference record). */
int oracle_measure(chp_t *t, int q, uint64_t seed, uint64_t shot, uint64_t midx, int force_zero) {
  int n = t->n;
  if (t->rows != 2 * n) return -1; /* a row subset cannot be measured */
  /* probabilistic iff some stabilizer has x_pq = 1; pivot = smallest */
  int p = -1;
  for (int i = n; i < 2 * n; ++i)
    if (XB(t, i, q)) { p = i; break; }
  if (p >= 0) {
    t->last_kind = 1;
    /* 1. make every other anticommuting generator commute: rowsum(i, p) */
    for (int i = 0; i < 2 * n; ++i)
      if (i != p && i != p - n && XB(t, i, q)) rowsum(t, i, p);
    /* 2. D_{p-n} <- S_p */
    memcpy(&XB(t, p - n, 0), &XB(t, p, 0), (size_t)n);
    memcpy(&ZB(t, p - n, 0), &ZB(t, p, 0), (size_t)n);
    t->r[p - n] = t->r[p];
    /* 3. S_p <- (-1)^m Z_q with a fresh coin m; return m */
    memset(&XB(t, p, 0), 0, (size_t)n);
    memset(&ZB(t, p, 0), 0, (size_t)n);
    ZB(t, p, q) = 1;
    int m = force_zero ? 0 : oracle_coin(seed, shot, midx);
    t->r[p] = (uint8_t)m;
    return m;
  }
  /* deterministic: (-1)^m Z_q = product of S_i over i with x_iq(D_i) = 1 */
  t->last_kind = 0;
  int s = 2 * n;
  memset(&XB(t, s, 0), 0, (size_t)n);
  memset(&ZB(t, s, 0), 0, (size_t)n);
  t->r[s] = 0;
  for (int i = 0; i < n; ++i)
    if (XB(t, i, q)) rowsum(t, s, i + n);
  for (int j = 0; j < n; ++j)
    if (XB(t, s, j) != 0 || ZB(t, s, j) != (j == q)) { t->det_check_fail++; break; }
  return t->r[s];
}

/* Runs a measurement list in order; record indices start at midx0. */
void oracle_measure_many(chp_t *t, const uint32_t *qubits, long count, uint64_t seed,
                         uint64_t shot, uint64_t midx0, int force_zero, uint8_t *out,
                         uint8_t *kind) {
  for (long i = 0; i < count; ++i) {
    out[i] = (uint8_t)oracle_measure(t, (int)qubits[i], seed, shot, midx0 + (uint64_t)i, force_zero);
    if (kind) kind[i] = (uint8_t)t->last_kind;
  }
}

/* ------------------------------------------------------------------ */
/* Pauli-frame sampling, Sec. 5 (Alg. 9)                                */
/* ------------------------------------------------------------------ */

/* One frame per shot: fx, fz are shots*n bytes (shot-major). Gates act on
 * the frame bits by the same rules as the tableau, without signs. */
static void frame_gate(uint8_t *fx, uint8_t *fz, int type, int a, int b) {
  uint8_t t8;
  switch (type) {
    case G_H: t8 = fx[a]; fx[a] = fz[a]; fz[a] = t8; break;
    case G_S: case G_SDG: fz[a] ^= fx[a]; break;
    case G_CX: fx[b] ^= fx[a]; fz[a] ^= fz[b]; break;
    case G_CZ: frame_gate(fx, fz, G_H, b, 0); frame_gate(fx, fz, G_CX, a, b); frame_gate(fx, fz, G_H, b, 0); break;
    case G_CY: frame_gate(fx, fz, G_S, b, 0); frame_gate(fx, fz, G_CX, a, b); frame_gate(fx, fz, G_S, b, 0); break;
    case G_SWAP:
      t8 = fx[a]; fx[a] = fx[b]; fx[b] = t8;
      t8 = fz[a]; fz[a] = fz[b]; fz[b] = t8; break;
    case G_ISWAP:
      frame_gate(fx, fz, G_CZ, a, b); frame_gate(fx, fz, G_SWAP, a, b);
      frame_gate(fx, fz, G_S, a, 0); frame_gate(fx, fz, G_S, b, 0); break;
    default: break; /* I, X, Y, Z change no frame bit */
  }
}

enum { N_X, N_Y, N_Z, N_DEP1, N_DEP2 };

/* Pauli code 0 = I, 1 = X, 2 = Y, 3 = Z on the frame of qubit q */
static void frame_pauli(uint8_t *fx, uint8_t *fz, int q, int code) {
  if (code == 1 || code == 2) fx[q] ^= 1u;
  if (code == 2 || code == 3) fz[q] ^= 1u;
}

/* noise op e with targets t[0..cnt) (pairs for DEPOLARIZE2), shot s */
static void frame_noise(uint8_t *fx, uint8_t *fz, int kind, double p, const uint32_t *t, long cnt,
                        uint64_t e, uint64_t seed, uint64_t s) {
  const uint64_t thr = oracle_noise_threshold(p);
  const long targets = kind == N_DEP2 ? cnt / 2 : cnt;
  for (long i = 0; i < targets; ++i) {
    uint64_t u, v;
    oracle_noise_draw(seed, e, (uint64_t)i, s, &u, &v);
    int fire = u < thr; /* thr = 2^32 when p >= 1 */
    if (!fire) continue;
    switch (kind) {
      case N_X: frame_pauli(fx, fz, (int)t[i], 1); break;
      case N_Y: frame_pauli(fx, fz, (int)t[i], 2); break;
      case N_Z: frame_pauli(fx, fz, (int)t[i], 3); break;
      case N_DEP1: frame_pauli(fx, fz, (int)t[i], 1 + (int)mul_hi(v, 3)); break;
      case N_DEP2: {
        int idx = 1 + (int)mul_hi(v, 15);
        frame_pauli(fx, fz, (int)t[2 * i], idx >> 2);
        frame_pauli(fx, fz, (int)t[2 * i + 1], idx & 3);
        break;
      }
      default: break;
    }
  }
}

/*
 * Samples `shots` shots of a program given as a list of ops:
 *   op_kind[o] = 0: apply gates[op_a[o] .. op_b[o]) (rows of 3 uint32)
 *   op_kind[o] = 1: measure qubits[op_a[o] .. op_b[o]) in order
 *   op_kind[o] = 2: noise channel noise_kind[o] with probability noise_p[o]
 *                   on the targets qubits[op_a[o] .. op_b[o])
 * ref[m] is the reference outcome of measurement m (program order).
 * out[m * shots + s] = outcome bit of measurement m in shot s.
 * Frame init: fx = 0, fz[q] = bit (s mod 64) of frame_word(seed, 0, q, s/64);
 * after measurement m of q: fz[q] = bit of frame_word(seed, m + 1, q, s/64).
 */
int oracle_frames(int n, const uint32_t *gates, const uint32_t *qubits, const int *op_kind,
                  const long *op_a, const long *op_b, const int *noise_kind, const double *noise_p,
                  long n_ops, const uint8_t *ref, long shots, uint64_t seed, uint8_t *out) {
  uint8_t *fx = (uint8_t *)calloc((size_t)n, 1), *fz = (uint8_t *)calloc((size_t)n, 1);
  if (!fx || !fz) { free(fx); free(fz); return -1; }
  for (long s = 0; s < shots; ++s) {
    uint64_t j = (uint64_t)s >> 6, bit = (uint64_t)s & 63u;
    for (int q = 0; q < n; ++q) {
      fx[q] = 0;
      fz[q] = (uint8_t)((oracle_frame_word(seed, 0, (uint64_t)q, j) >> bit) & 1u);
    }
    long m = 0;
    uint64_t e = 0; /* noise ops so far */
    for (long o = 0; o < n_ops; ++o) {
      if (op_kind[o] == 0) {
        for (long g = op_a[o]; g < op_b[o]; ++g)
          frame_gate(fx, fz, (int)gates[3 * g], (int)gates[3 * g + 1], (int)gates[3 * g + 2]);
      } else if (op_kind[o] == 2) {
        frame_noise(fx, fz, noise_kind[o], noise_p[o], qubits + op_a[o], op_b[o] - op_a[o], e++, seed,
                    (uint64_t)s);
      } else {
        for (long i = op_a[o]; i < op_b[o]; ++i, ++m) {
          int q = (int)qubits[i];
          out[(size_t)m * (size_t)shots + (size_t)s] = (uint8_t)(fx[q] ^ ref[m]);
          fz[q] = (uint8_t)((oracle_frame_word(seed, (uint64_t)m + 1, (uint64_t)q, j) >> bit) & 1u);
        }
      }
    }
  }
  free(fx); free(fz);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Inverse tableau with qubit-indexed signs: the representation of the  */
/* paper's measurement variant (Sec. 3.2, Alg. 1; Stim's TableauSimulator) */
/* ------------------------------------------------------------------ */
/*
 * For the Clifford C that prepares the state from |0...0>, this mode keeps
 * the Pauli strings C^dag Z_q C and C^dag X_q C over the input qubits, one per
 * qubit q, each with a sign. Their bits are the bits of the extended tableau
 * of Sec. 2.5 read by columns. With XS[i][q] the x bit of stabilizer i at
 * qubit q (row n + i of x), XD[i][q] the x bit of destabilizer i (row i of
 * x), and ZS, ZD the same for z,
 *   C^dag Z_q C = (-1)^ss[q] * prod_i sigma(XS[i][q], XD[i][q])   (x, z at input i)
 *   C^dag X_q C = (-1)^sd[q] * prod_i sigma(ZS[i][q], ZD[i][q]).
 * (C^dag P C anticommutes with Z_i iff P anticommutes with C Z_i C^dag =
 * stabilizer i, and with X_i iff P anticommutes with destabilizer i.) The
 * sign vectors S_S and S_D of Alg. 1 are ss and sd, indexed by qubit (the
 * paper's reading G2: these signs belong to the inverse tableau, not to the
 * forward generators).
 *
 * A gate G appended to the circuit turns C into G C, so every image becomes
 * that of G^dag P G: the bits follow the column rules of Eq. 4 (same bits as
 * the forward tableau), and the signs of the gate's qubits follow from the
 * phase of a product of two images. A measurement runs Alg. 1: pivot = the
 * smallest stabilizer index with XS[p][q] = 1; CX injections from the pivot
 * into every later anticommuting stabilizer (in index order); the pivot is
 * swapped for a commuting generator by an H or an H_YZ injection; an X
 * injection sets the outcome to the coin. A deterministic outcome is ss[q].
 */
typedef struct {
  int n;
  uint8_t *x, *z;   /* 2n rows of n bits, as in chp_t */
  uint8_t *ss, *sd; /* n sign bits each */
  int last_kind;    /* 1 = last measurement was probabilistic, 0 = deterministic */
  long odd_count;   /* products of images whose phase had the wrong parity (must stay 0) */
} inv_t;

#define IXB(t, i, j) ((t)->x[(size_t)(i) * (size_t)(t)->n + (size_t)(j)])
#define IZB(t, i, j) ((t)->z[(size_t)(i) * (size_t)(t)->n + (size_t)(j)])

void oracle_inv_reset(inv_t *t, const uint8_t *initstate) {
  int n = t->n;
  memset(t->x, 0, (size_t)(2 * n) * n);
  memset(t->z, 0, (size_t)(2 * n) * n);
  for (int i = 0; i < n; ++i) {
    IXB(t, i, i) = 1;     /* destabilizer i = X_i: C^dag Z_i C has z at input i */
    IZB(t, n + i, i) = 1; /* stabilizer i = Z_i: C^dag X_i C has x at input i */
    /* |1> on qubit i is X_i|0>: X_i Z_i X_i = -Z_i, X_i X_i X_i = X_i */
    t->ss[i] = (uint8_t)(initstate && initstate[i] ? 1 : 0);
    t->sd[i] = 0;
  }
  t->last_kind = -1;
  t->odd_count = 0;
}

inv_t *oracle_inv_new(int n) {
  fill_g_table();
  inv_t *t = (inv_t *)calloc(1, sizeof(inv_t));
  if (!t) return NULL;
  t->n = n;
  size_t cells = (size_t)(2 * n) * (size_t)(n > 0 ? n : 1);
  t->x = (uint8_t *)calloc(cells, 1);
  t->z = (uint8_t *)calloc(cells, 1);
  t->ss = (uint8_t *)calloc((size_t)n + 1, 1);
  t->sd = (uint8_t *)calloc((size_t)n + 1, 1);
  if (!t->x || !t->z || !t->ss || !t->sd) {
    free(t->x); free(t->z); free(t->ss); free(t->sd); free(t);
    return NULL;
  }
  oracle_inv_reset(t, NULL);
  return t;
}

void oracle_inv_free(inv_t *t) {
  if (!t) return;
  free(t->x); free(t->z); free(t->ss); free(t->sd); free(t);
}

/* x, z: 2n*n bytes (rows as in oracle_get); ss, sd: n bytes */
void oracle_inv_get(const inv_t *t, uint8_t *x, uint8_t *z, uint8_t *ss, uint8_t *sd) {
  size_t cells = (size_t)(2 * t->n) * t->n;
  memcpy(x, t->x, cells); memcpy(z, t->z, cells);
  memcpy(ss, t->ss, (size_t)t->n); memcpy(sd, t->sd, (size_t)t->n);
}

int oracle_inv_last_kind(const inv_t *t) { return t->last_kind; }
long oracle_inv_odd_count(const inv_t *t) { return t->odd_count; }

/* bits at input i of the image of X_q (w = 0) or Z_q (w = 1) */
static int img_x(const inv_t *t, int w, int q, int i) { return w ? IXB(t, t->n + i, q) : IZB(t, t->n + i, q); }
static int img_z(const inv_t *t, int w, int q, int i) { return w ? IXB(t, i, q) : IZB(t, i, q); }

/* image(P_a) * image(P_b) = i^e * sigma(bitwise sum); returns e mod 4 */
static int img_product_phase(const inv_t *t, int wa, int a, int wb, int b) {
  long e = 0;
  for (int i = 0; i < t->n; ++i)
    e += g_fn(img_x(t, wa, a, i), img_z(t, wa, a, i), img_x(t, wb, b, i), img_z(t, wb, b, i));
  return (int)(((e % 4) + 4) % 4);
}

/* H: H X H = Z and H Z H = X, so the two images of qubit a trade places
 * (bits: x_a <-> z_a in every row, Eq. 4) */
static void inv_h(inv_t *t, int a) {
  uint8_t s = t->ss[a];
  t->ss[a] = t->sd[a];
  t->sd[a] = s;
  for (int i = 0; i < 2 * t->n; ++i) {
    uint8_t x = IXB(t, i, a);
    IXB(t, i, a) = IZB(t, i, a);
    IZB(t, i, a) = x;
  }
}

/* S (dagger = 0) or S^dag (dagger = 1): S^dag X S = -Y and S X S^dag = Y with
 * Y = i X Z; Z is fixed. The new image of X_a is -i (resp. i) times
 * image(X_a) image(Z_a) (bits: z_a ^= x_a in every row). */
static void inv_s(inv_t *t, int a, int dagger) {
  int e = img_product_phase(t, 0, a, 1, a);
  int f = (e + (dagger ? 1 : 3)) & 3; /* times i (= i^1) or -i (= i^3) */
  if (f & 1) t->odd_count++;         /* the images of X_a and Z_a anticommute: e is odd */
  t->sd[a] = (uint8_t)(t->sd[a] ^ t->ss[a] ^ (f >> 1));
  for (int i = 0; i < 2 * t->n; ++i) IZB(t, i, a) ^= IXB(t, i, a);
}

/* CX (control c, target tq): X_c -> X_c X_t and Z_t -> Z_c Z_t under
 * conjugation; X_t and Z_c are fixed (bits: x_t ^= x_c, z_c ^= z_t). */
static void inv_cx(inv_t *t, int c, int tq) {
  int e1 = img_product_phase(t, 0, c, 0, tq); /* image(X_c) image(X_t), commuting: even */
  int e2 = img_product_phase(t, 1, c, 1, tq); /* image(Z_c) image(Z_t), commuting: even */
  if ((e1 | e2) & 1) t->odd_count++;
  t->sd[c] = (uint8_t)(t->sd[c] ^ t->sd[tq] ^ (e1 >> 1));
  t->ss[tq] = (uint8_t)(t->ss[tq] ^ t->ss[c] ^ (e2 >> 1));
  for (int i = 0; i < 2 * t->n; ++i) {
    IXB(t, i, tq) ^= IXB(t, i, c);
    IZB(t, i, c) ^= IZB(t, i, tq);
  }
}

void oracle_inv_gate(inv_t *t, int type, int a, int b) {
  switch (type) {
    case G_I: break;
    case G_X: t->ss[a] ^= 1u; break;                /* X Z X = -Z */
    case G_Z: t->sd[a] ^= 1u; break;                /* Z X Z = -X */
    case G_Y: t->ss[a] ^= 1u; t->sd[a] ^= 1u; break; /* Y anticommutes with X and Z */
    case G_H: inv_h(t, a); break;
    case G_S: inv_s(t, a, 0); break;
    case G_SDG: inv_s(t, a, 1); break;
    case G_CX: inv_cx(t, a, b); break;
    case G_CZ: inv_h(t, b); inv_cx(t, a, b); inv_h(t, b); break;
    case G_CY: inv_s(t, b, 1); inv_cx(t, a, b); inv_s(t, b, 0); break;
    case G_SWAP: inv_cx(t, a, b); inv_cx(t, b, a); inv_cx(t, a, b); break;
    case G_ISWAP:
      oracle_inv_gate(t, G_CZ, a, b); oracle_inv_gate(t, G_SWAP, a, b);
      inv_s(t, a, 0); inv_s(t, b, 0); break;
    default: break;
  }
}

void oracle_inv_apply(inv_t *t, const uint32_t *gates, long count) {
  for (long g = 0; g < count; ++g)
    oracle_inv_gate(t, (int)gates[3 * g], (int)gates[3 * g + 1], (int)gates[3 * g + 2]);
}

/* Alg. 1's injections, element by element over the n qubit positions of the
 * rows they are given (s: a sign vector indexed by qubit). */
static void inject_cx(int n, uint8_t *s, const uint8_t *xc, uint8_t *zc, uint8_t *xt, const uint8_t *zt) {
  for (int j = 0; j < n; ++j) {
    s[j] ^= (uint8_t)(xc[j] & zt[j] & ((zc[j] ^ xt[j]) ^ 1u));
    xt[j] ^= xc[j];
    zc[j] ^= zt[j];
  }
}

static void inject_invp(int n, uint8_t *s, uint8_t *x, const uint8_t *z) {
  for (int j = 0; j < n; ++j) {
    s[j] ^= (uint8_t)(x[j] & (z[j] ^ 1u));
    x[j] ^= z[j];
  }
}

static void inject_had(int n, uint8_t *s, uint8_t *x, uint8_t *z) {
  for (int j = 0; j < n; ++j) {
    s[j] ^= (uint8_t)(x[j] & z[j]);
    uint8_t v = x[j];
    x[j] = z[j];
    z[j] = v;
  }
}

static void inject_x(int n, uint8_t *s, const uint8_t *z) {
  for (int j = 0; j < n; ++j) s[j] ^= z[j];
}

/* Z-measurement of qubit q (Alg. 1, ProbabilisticMeasurement); the coin is
 * coin(seed, shot, midx). Rows: XS[i] = x row n + i, XD[i] = x row i, ZS[i]
 * = z row n + i, ZD[i] = z row i. */
int oracle_inv_measure(inv_t *t, int q, uint64_t seed, uint64_t shot, uint64_t midx) {
  int n = t->n;
  int p = -1;
  for (int i = 0; i < n; ++i)
    if (IXB(t, n + i, q)) { p = i; break; }
  if (p < 0) {
    t->last_kind = 0;
    return t->ss[q];
  }
  t->last_kind = 1;
  uint8_t *XSp = &IXB(t, n + p, 0), *XDp = &IXB(t, p, 0), *ZSp = &IZB(t, n + p, 0), *ZDp = &IZB(t, p, 0);
  /* GE: CX injections from the pivot into the later anticommuting stabilizers, in order */
  for (int tg = p + 1; tg < n; ++tg) {
    if (!IXB(t, n + tg, q)) continue;
    inject_cx(n, t->sd, ZSp, ZDp, &IZB(t, n + tg, 0), &IZB(t, tg, 0));
    inject_cx(n, t->ss, XSp, XDp, &IXB(t, n + tg, 0), &IXB(t, tg, 0));
  }
  /* swap the anticommuting stabilizer for a commuting one: the Y case takes
   * H_YZ (InvP), the X case H */
  if (XDp[q]) {
    inject_invp(n, t->sd, ZSp, ZDp);
    inject_invp(n, t->ss, XSp, XDp);
  } else {
    inject_had(n, t->sd, ZSp, ZDp);
    inject_had(n, t->ss, XSp, XDp);
  }
  /* the outcome is the coin: an X injection on the pivot flips it if needed */
  int m = oracle_coin(seed, shot, midx);
  if (t->ss[q] != (uint8_t)m) {
    inject_x(n, t->sd, ZDp);
    inject_x(n, t->ss, XDp);
  }
  return t->ss[q];
}

void oracle_inv_measure_many(inv_t *t, const uint32_t *qubits, long count, uint64_t seed,
                             uint64_t shot, uint64_t midx0, uint8_t *out, uint8_t *kind) {
  for (long i = 0; i < count; ++i) {
    out[i] = (uint8_t)oracle_inv_measure(t, (int)qubits[i], seed, shot, midx0 + (uint64_t)i);
    if (kind) kind[i] = (uint8_t)t->last_kind;
  }
}
