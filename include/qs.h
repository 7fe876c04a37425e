/*
 * qs.h - C ABI of the GB300 stabilizer-tableau simulator (libqs.so).
 *
 * The library simulates Clifford circuits with Z-measurements on one GPU
 * (sm_103a) by Aaronson-Gottesman tableau evolution over a bit-packed
 * X/Z/sign tableau, following arXiv 2603.14641 ("QuaSARQ"):
 *   - extended tableau (n destabilizers D_i, n stabilizers S_i), Sec. 2.5 Eq. 7;
 *   - gate layers by the column update rules of Sec. 2.4 Eq. 4, applied to all
 *     2n rows word-parallel (Sec. 4.4, Alg. 3);
 *   - projective Z-measurement by CHP (Sec. 2.5): pivot search, rowsum of the
 *     pivot into every anticommuting row with the mod-4 phase, and the
 *     deterministic-outcome product (Sec. 2.5, Sec. 3.2 Eqs. 9-11);
 *   - many-shot Pauli-frame sampling (Sec. 5, Alg. 9).
 *
 * Conventions for every call:
 *   - Return value: QS_OK (0) or a negative QS_ERR_* code; qs_last_error()
 *     gives a message for the calling thread. No C++ exception crosses the ABI.
 *   - Host arrays are owned by the caller and are read (or written) before the
 *     call returns, except where a call says otherwise.
 *   - Device memory is owned by the caller when it passes a workspace, else by
 *     the library (cudaMalloc at create, cudaFree at destroy).
 *   - All device work is ordered on the stream given at create. Calls that
 *     return host data synchronise that stream; the others do not.
 *   - A sim is used by one host thread at a time.
 *   - On QS_ERR_ARG / QS_ERR_SIZE the sim is unchanged. After QS_ERR_CUDA or
 *     QS_ERR_INTERNAL the sim is flagged unusable and later calls fail with
 *     QS_ERR_STATE.
 */
#ifndef QS_GB300_API_H_
#define QS_GB300_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QS_OK 0
#define QS_ERR_ARG (-1)      /* bad argument: qubit >= n, overlapping qubits in a layer, unknown gate */
#define QS_ERR_OOM (-2)      /* device or host allocation failed */
#define QS_ERR_CUDA (-3)     /* a CUDA call failed */
#define QS_ERR_TIMEOUT (-4)  /* a bounded device wait ran out */
#define QS_ERR_SIZE (-5)     /* output buffer too small or capacity exceeded */
#define QS_ERR_STATE (-6)    /* the sim is unusable after an earlier device error */
#define QS_ERR_INTERNAL (-7) /* a device self-check failed (odd rowsum phase, bad deterministic product) */

/* Gate types: the paper's 11-gate Clifford set (Sec. 6 "Benchmarks") plus identity. */
enum {
  QS_I = 0, QS_X = 1, QS_Y = 2, QS_Z = 3, QS_H = 4, QS_S = 5, QS_SDG = 6,
  QS_CX = 7, QS_CY = 8, QS_CZ = 9, QS_SWAP = 10, QS_ISWAP = 11, QS_NUM_GATE_TYPES = 12,
  QS_MEASURE = 12 /* operation type of qs_schedule_windows only: Z-measurement of q0 */
};

/* One gate record. q1 is ignored for one-qubit gates; for CX/CY q0 is the
 * control and q1 the target. */
typedef struct qs_gate {
  uint32_t type;
  uint32_t q0;
  uint32_t q1;
} qs_gate;

/* Key of the counter-based random source (Philox4x64-10, Salmon et al. 2011;
 * the paper draws Philox numbers through cuRAND, Sec. 5). The coin of the
 * probabilistic outcome with record index m is bit 0 of word 0 of
 * Philox(counter = (m, shot, 0, 0), key = (seed, 0x51A7E)). */
typedef struct qs_key {
  uint64_t seed;
  uint64_t shot;
} qs_key;

typedef struct qs_options {
  uint64_t record_capacity; /* max measurements kept in the device record; 0 = 16 n + 65536 */
  uint32_t flags;           /* QS_FLAG_* bits, 0 for defaults */
  uint32_t reserved;
} qs_options;

/* qs_options.flags: apply every device-resident layer with its own kernel
 * instead of fusing a run of layers into one shared-memory pass (the fused
 * pass is used for n <= 14,080; results are identical either way). */
#define QS_FLAG_NO_FUSION 1u
/* qs_options.flags: run every measurement as five separate launches (gather,
 * rowsum, deterministic partials, combine, finalize) instead of the pipelined
 * two launches per measurement; results are identical either way. */
#define QS_FLAG_UNPIPELINED_MEASURE 2u
/* qs_options.flags: never measure in blocks. By default a window of >= 16
 * measurements on >= 64 qubits is measured in blocks of up to 64 with one
 * pass over the tableau per block (identical results); the blocked path waits
 * for the stream once per block. */
#define QS_FLAG_NO_BLOCKED_MEASURE 4u
/* qs_options.flags: address the row-major tableau with 64-bit word offsets in
 * the blocked measurement's apply pass even when 32-bit ones suffice. By
 * default 64-bit offsets are used only when the row-major matrix holds 2^32
 * words or more (about 371,000 qubits and up); the flag runs that code path on
 * a tableau of any size (identical results). */
#define QS_FLAG_WIDE_OFFSETS 8u
/* qs_options.flags: run the blocked measurement's symbolic pass (which rows
 * each of a block's measurements targets) as one launch per measurement over
 * every row. By default that launch sequence is used only above 25,600 qubits;
 * up to that size one CTA runs every step over the stabilizer rows held in
 * shared memory. The flag runs the large-size code path at any size
 * (identical results). */
#define QS_FLAG_STEP_SYMBOLIC 16u
/* qs_options.flags: inverse-tableau mode, the representation of the paper's
 * own measurement variant (Sec. 3.2, Alg. 1: Gaussian elimination by CX
 * injection, as in Stim). For the Clifford C that prepares the state from
 * |0...0>, the sim keeps C^dag Z_q C and C^dag X_q C with qubit-indexed
 * signs S_S[q] and S_D[q] (qs_sim_qubit_signs). The tableau bits are those
 * of the default (CHP) mode under gates, read by columns; per-row signs are
 * not kept (exports give 0 there). Measurements run Alg. 1 (pivot = smallest
 * anticommuting stabilizer, CX injections into the later ones, an H or H_YZ
 * and an X injection on the pivot), four launches each; records and
 * measurement kinds equal the CHP mode's under the same keys, and the state
 * is the same, though the tableau bits after a measurement differ. Layers
 * run one launch each (no fused segments); measurements are never blocked;
 * qs_sim_tableau_import is refused. Fixed at create. */
#define QS_FLAG_INVERSE_TABLEAU 32u

typedef struct qs_sim qs_sim;

/* Layouts for qs_sim_tableau_export and qs_sim_tableau_import. */
enum {
  /* Rows 0..2n-1 (destabilizers, then stabilizers), each ceil(n/64)
   * x-words then ceil(n/64) z-words (bit j of word w = qubit 64 w + j),
   * followed by ceil(2n/64) sign words (bit i = sign of row i). */
  QS_LAYOUT_ROWS_PACKED = 0,
  /* The device's own column-major layout (the one gate layers run on, Sec. 4.1),
   * copied without repacking. With k = ceil(n/64) and W = 4 ceil(k/2) (2k
   * rounded up to a multiple of 4): n X columns of W words (column of qubit q
   * at word q W), then n Z columns of W words, then W sign words. Bit g of a
   * column or of the sign words belongs to generator g in packed numbering:
   * destabilizer i at g = i, stabilizer i at g = 64 k + i; every other bit is
   * zero. (2n + 1) W words in all. */
  QS_LAYOUT_NATIVE = 1
};

/* Library version string. */
const char *qs_version(void);

/* Message for the last error on the calling thread ("" if none). */
const char *qs_last_error(void);

/* Device bytes a sim of n qubits needs when the caller supplies the workspace
 * (tableau in column- and row-major form, scratch and record). */
size_t qs_sim_required_bytes(uint32_t n, const qs_options *opt);

/*
 * Creates a sim of n >= 1 qubits in state |0...0> (Sec. 4.1 Alg. 2,
 * AllocateTableau + InitializeTableau).
 *   opt:        NULL for defaults.
 *   cuda_stream: cudaStream_t the sim enqueues on (NULL = legacy default).
 *   workspace:  device pointer of >= qs_sim_required_bytes(n, opt) bytes,
 *               256-byte aligned, owned by the caller and kept alive until
 *               qs_sim_destroy; or NULL to let the library cudaMalloc it.
 * Errors: QS_ERR_ARG (n == 0 or n > 2^20, unaligned workspace),
 * QS_ERR_SIZE (workspace too small), QS_ERR_OOM, QS_ERR_CUDA.
 */
int qs_sim_create(uint32_t n, const qs_options *opt, void *cuda_stream, void *workspace,
                  size_t workspace_bytes, qs_sim **out);

/* Waits for the sim's stream, frees what the library allocated. NULL is a no-op. */
int qs_sim_destroy(qs_sim *sim);

/* Re-initialises the tableau to a computational basis state (Alg. 2 input
 * initstate): D_i = X_i, S_i = Z_i, and both rows of qubit i get sign
 * initstate[i] (Sec. 2.5 Eq. 8 pattern). initstate: n bytes (0/1) on the
 * host, or NULL for |0...0>. Clears the record and the op log. */
int qs_sim_reset(qs_sim *sim, const uint8_t *initstate);

/*
 * Applies one layer of gates on pairwise disjoint qubits (a window of
 * Sec. 4.2) to every tableau row (Sec. 2.4 Eq. 4; Sec. 4.4 Alg. 3).
 * gates: host array of n_gates records. Validated on the host before any
 * device work: QS_ERR_ARG for an unknown type, a qubit >= n, q0 == q1 on a
 * two-qubit gate, or a qubit used twice in the layer. The layer is kept in
 * the sim's op log for qs_sim_sample.
 */
int qs_sim_apply_layer(qs_sim *sim, const qs_gate *gates, uint32_t n_gates);

/*
 * Validates and packs layered gates into the device record format used by
 * qs_sim_apply_layers_dev: 2 uint32 per gate, (type << 24 | q0, q1).
 *   gates:     host records, layer l = gates[layer_ptr[l] .. layer_ptr[l+1]).
 *   layer_ptr: host array of n_layers + 1 nondecreasing offsets, layer_ptr[0] = 0.
 *   packed:    host output of 2 * layer_ptr[n_layers] uint32.
 * Errors: QS_ERR_ARG as qs_sim_apply_layer (message names the layer/gate).
 */
int qs_pack_layers(uint32_t n, const qs_gate *gates, const int64_t *layer_ptr, uint32_t n_layers,
                   uint32_t *packed);

/*
 * Applies layers l_begin..l_end-1 of a circuit already resident in device
 * memory (packed by qs_pack_layers for this n and copied to the device by the
 * caller). packed_dev must stay valid until the work has run and, if
 * qs_sim_sample will replay it, until the sim is reset or destroyed.
 * layer_ptr: host offsets as given to qs_pack_layers (layer l of the call is
 *            packed_dev gate records [layer_ptr[l], layer_ptr[l+1])).
 * Errors: QS_ERR_ARG (NULL argument, l_end < l_begin, a negative or
 * decreasing offset, a layer of more than n gates); gate records that are
 * invalid on the device are skipped and raise QS_ERR_INTERNAL at the next sync.
 */
int qs_sim_apply_layers_dev(qs_sim *sim, const uint32_t *packed_dev, const int64_t *layer_ptr,
                            uint32_t l_begin, uint32_t l_end);

/*
 * Measures qubits in the Z basis, one after another in array order (CHP,
 * Sec. 2.5; measurement indices continue the sim's record). Each outcome is
 * appended to the device record. Probabilistic outcomes are the keyed coin of
 * the measurement's record index; deterministic outcomes follow from the
 * stabilizer group (Sec. 2.5 Eq. 6).
 *   qubits:   host array of count qubit indices (< n; repeats allowed).
 *   outcomes: host array of count bytes to receive the outcomes (0/1), or
 *             NULL to leave them on the device (no synchronisation).
 * Errors: QS_ERR_ARG (qubit >= n), QS_ERR_SIZE (record capacity exceeded).
 */
int qs_sim_measure(qs_sim *sim, const uint32_t *qubits, uint32_t count, qs_key key,
                   uint8_t *outcomes);

/* As qs_sim_measure with the qubit list already in device memory (count
 * uint32, each < n; not checked on the host: an out-of-range qubit makes the
 * kernels skip the measurement and raise QS_ERR_INTERNAL at the next sync).
 * The list must stay valid until qs_sim_sample if that will replay it. */
int qs_sim_measure_dev(qs_sim *sim, const uint32_t *qubits_dev, uint32_t count, qs_key key);

/* Number of measurements in the record. */
uint64_t qs_sim_num_measurements(const qs_sim *sim);

/* Copies record entries [first, first + count) to host bytes (0/1). Syncs. */
int qs_sim_record(qs_sim *sim, uint64_t first, uint64_t count, uint8_t *dst);

/* Kind of each record entry [first, first + count) as host bytes: 1 = the
 * outcome was probabilistic (a pivot existed, the outcome is the coin), 0 =
 * deterministic (Sec. 2.5), 2 = restored by qs_sim_tableau_import. Syncs. */
int qs_sim_record_kinds(qs_sim *sim, uint64_t first, uint64_t count, uint8_t *dst);

/* Pauli noise channels of qs_sim_noise (the values are part of the ABI). */
enum {
  QS_NOISE_X = 0,           /* X with probability p */
  QS_NOISE_Y = 1,           /* Y with probability p */
  QS_NOISE_Z = 2,           /* Z with probability p */
  QS_NOISE_DEPOLARIZE1 = 3, /* X, Y or Z, each with probability p/3 */
  QS_NOISE_DEPOLARIZE2 = 4, /* one of the 15 non-identity two-qubit Paulis, each p/15 */
  QS_NUM_NOISE_KINDS = 5
};

/*
 * Appends a Pauli noise channel to the sim's op log. Noise acts on the shots
 * qs_sim_sample draws, through the Pauli frames (Sec. 3: frames carry error
 * events as well as measurement randomness, so one noiseless reference shot
 * serves every noisy shot); the tableau and the single-shot record are not
 * touched. The paper fixes no channel set; these are the usual ones.
 *   kind:    QS_NOISE_*.
 *   p:       probability in [0, 1].
 *   targets: host array of count qubits (< n, pairwise distinct); for
 *            QS_NOISE_DEPOLARIZE2, count is even and targets hold pairs
 *            (targets[2i], targets[2i+1]). Copied before the call returns.
 * Randomness: for target i (pair i for DEPOLARIZE2) of noise op e (numbered
 * from 0 in the op log) and shot s, the channel fires iff p >= 1 or
 * u < floor(p * 2^32), where bit 31 - k of u (k = 0..31) is bit (s & 63) of
 * word (k & 3) of Philox4x64-10(counter = (e, i, 8 (s >> 6) + (k >> 2), 3),
 * key = (seed, 0xE5505)). When it fires, v = word 0 of
 * Philox4x64-10(counter = (e, i, s, 4), same key) picks the Pauli:
 * DEPOLARIZE1 applies 1 + floor(3 v / 2^64) (1 = X, 2 = Y, 3 = Z) and
 * DEPOLARIZE2 the pair with index 1 + floor(15 v / 2^64) = 4 a + b
 * (0 = I, 1 = X, 2 = Y, 3 = Z on the first and second target).
 * Errors: QS_ERR_ARG (unknown kind, p outside [0, 1] or NaN, a target >= n
 * or repeated, odd count for DEPOLARIZE2). No device work.
 */
int qs_sim_noise(qs_sim *sim, int kind, double p, const uint32_t *targets, uint32_t count);

/* Device bytes of frame workspace qs_sim_sample needs for `shots` shots. */
size_t qs_sim_sample_required_bytes(const qs_sim *sim, uint64_t shots);

/*
 * Samples `shots` shots of the program in the sim's op log (every layer,
 * measurement and noise channel since create/reset) by Pauli frames (Sec. 5,
 * Alg. 9): frames
 * start with X~ = 0, Z~ = keyed Philox words; gate layers act on the frames
 * without signs; measurement m of qubit q outputs X~[q] XOR ref[m] and
 * re-randomises Z~[q]. The reference ref is the sim's own single-shot record.
 * Frame words: word j (shots 64 j .. 64 j + 63) of qubit q after event e is
 * word (j & 3) of Philox(counter = (e, q, j >> 2, 1), key = (seed, 0xF4A3E)),
 * e = 0 at initialisation and e = m + 1 after measurement m.
 *   shots:  1 .. 2e9 (QS_ERR_ARG otherwise).
 *   record: [M][ceil(shots/64)] uint64 (M = qs_sim_num_measurements), bit s of
 *           word j of measurement m = outcome of shot 64 j + s (bits >= shots
 *           are 0); host or device pointer; record_words >= M * ceil(shots/64).
 *   frame_ws: device workspace of >= qs_sim_sample_required_bytes bytes, or
 *           NULL to let the library allocate it for the call.
 * Syncs the stream when record is a host pointer.
 */
int qs_sim_sample(qs_sim *sim, uint64_t shots, uint64_t seed, uint64_t *record,
                  size_t record_words, void *frame_ws, size_t frame_ws_bytes);

/*
 * Copies the tableau out in `layout` (QS_LAYOUT_ROWS_PACKED or
 * QS_LAYOUT_NATIVE) to host or device memory (told apart by unified
 * addressing). needed: if not NULL, receives the byte size. dst may be NULL
 * to query. NATIVE needs no repacking on the host, only the layout switch
 * back to columns when the last operation was a measurement.
 * Errors: QS_ERR_ARG (unknown layout), QS_ERR_SIZE (dst_bytes too small). Syncs.
 */
int qs_sim_tableau_export(qs_sim *sim, int layout, void *dst, size_t dst_bytes, size_t *needed);

/*
 * Restores a checkpoint (the paper has none; tableau, record and keys make one
 * because the coins are keyed by record index): the tableau from a host
 * buffer in one of qs_sim_tableau_export's layouts and the first
 * record_count record entries (0/1 bytes, host). Measurements after the import continue the
 * record at index record_count, so with the same keys they reproduce the
 * uninterrupted run bit for bit. The op log is cleared and qs_sim_sample is
 * refused (QS_ERR_STATE) until qs_sim_reset: frame sampling replays the
 * program from |0...0>. The tableau is not checked for validity beyond its
 * padding bits (past qubit n - 1 in ROWS_PACKED, outside the packed generator
 * numbering in NATIVE), which must be zero (QS_ERR_ARG). Syncs.
 * Errors: QS_ERR_ARG (layout, padding bits, NULL record), QS_ERR_SIZE
 * (src_bytes too small, record_count above the record capacity).
 */
int qs_sim_tableau_import(qs_sim *sim, int layout, const void *src, size_t src_bytes,
                          const uint8_t *record, uint64_t record_count);

/*
 * Copies selected generator rows to host memory: rows[i] in 0..2n-1
 * (0..n-1 destabilizers D_i, n..2n-1 stabilizers S_i, Sec. 2.5 Eq. 7). For
 * each row dst receives ceil(n/64) x-words, ceil(n/64) z-words (bit j of word
 * w = qubit 64 w + j) and one word with the sign bit in bit 0, i.e.
 * count * (2 ceil(n/64) + 1) words. Syncs.
 * Errors: QS_ERR_ARG (row >= 2n or NULL pointers).
 */
int qs_sim_export_rows(qs_sim *sim, const uint32_t *rows, uint32_t count, uint64_t *dst);

/*
 * Inverse-tableau mode only (QS_FLAG_INVERSE_TABLEAU): copies the qubit-indexed
 * signs of Alg. 1 to dst (host or device): ceil(n/64) words of S_S (bit q of
 * word q / 64 = sign of C^dag Z_q C), then ceil(n/64) words of S_D (sign of
 * C^dag X_q C). dst_words >= 2 ceil(n/64). Syncs.
 * Errors: QS_ERR_ARG (NULL dst), QS_ERR_SIZE, QS_ERR_STATE (the sim is in
 * the default mode).
 */
int qs_sim_qubit_signs(qs_sim *sim, uint64_t *dst, size_t dst_words);

/* Waits for the stream and checks the device error flags:
 * QS_ERR_INTERNAL if a self-check failed, QS_ERR_TIMEOUT if a bounded wait
 * ran out. */
int qs_sim_sync(qs_sim *sim);

/*
 * Allocation-free variant of qs_sim_sample (the paper has no counterpart).
 * For callers that cannot allocate device memory when they sample -- a
 * serving process that reserved the GPU's memory for its own pool up front, a
 * framework whose caching allocator must own every device byte, or a
 * latency-critical loop that cannot afford cudaFree's device-wide
 * synchronisation -- the frames are kept in one file-scope device array of
 * QS_NOALLOC_SCRATCH_BYTES (32 MiB) inside libqs instead of a workspace.
 * Output and sampling rule are those of qs_sim_sample; the call itself
 * allocates nothing (no cudaMalloc/cudaFree, no allocating library routine).
 *   record: host or device pointer of >= M * ceil(shots/64) words.
 * Limits and behaviour:
 *   - 2 * n * ceil(ceil(shots/64)/4)*4 * 8 bytes of frames (each rounded up to
 *     256) plus M * ceil(shots/64) * 8 bytes must fit in the array, else
 *     QS_ERR_SIZE with the sizes in qs_last_error().
 *   - The array is placed on a device, and its address looked up, when the
 *     first sim is created there (qs_sim_create, with that device current), so a
 *     process that creates its sims before it reserves the rest of the GPU for
 *     its own pool has the array in place; from then on that GPU holds it until
 *     the process exits. If that set-up failed at create (the sim itself is
 *     fine), the first qs_sim_sample_noalloc on the device tries again and, if it
 *     fails, returns QS_ERR_CUDA without marking the sim unusable.
 *   - All calls share the array and each call starts by clearing it (X~ = 0,
 *     Z~ rewritten); two calls whose work overlaps on the GPU (different
 *     streams, or different sims on one device) race on it. Calls from several
 *     host threads are serialised on the host, not on the GPU.
 *   - When the set-up is left to the first qs_sim_sample_noalloc on a device
 *     (create could not do it), make that first call before any stream capture.
 */
#define QS_NOALLOC_SCRATCH_BYTES (32u << 20)
int qs_sim_sample_noalloc(qs_sim *sim, uint64_t shots, uint64_t seed, uint64_t *record,
                          size_t record_words);

/* ---------------------------------------------------------------------- */
/* Batched persistent launch: many independent circuits, one kernel launch */
/* ---------------------------------------------------------------------- */

/*
 * One circuit of a batch, as a program of rounds: round r applies layers
 * [round_layers[r], round_layers[r+1]) (each layer a window of gates on
 * disjoint qubits, Sec. 4.2) and then measures, in order,
 * qubits[round_meas[r] .. round_meas[r+1]) in the Z basis (CHP, Sec. 2.5).
 * The coin of the circuit's m-th measurement (program order) is keyed by
 * (seed, shot, m) exactly as in qs_sim_measure, so a circuit's record and
 * tableau are the same alone (qs_sim_*) and in a batch. All arrays are host
 * memory and are copied at qs_batch_create. 1 <= n <= 2^20.
 *
 * Circuits of n < 1024 qubits run in one cooperative persistent kernel on the
 * batch's stream (their cost is per-launch overhead when they run alone);
 * circuits of n >= 1024 run through one qs_sim each (blocked measurement),
 * spread over up to 16 worker streams that host threads drive during
 * qs_batch_run. The paper has no batch mode; this follows the batched
 * workload's shape (many small and some large circuits).
 */
typedef struct qs_batch_circuit {
  uint32_t n;
  uint32_t n_layers;
  const qs_gate *gates;          /* layer l = gates[layer_ptr[l] .. layer_ptr[l+1]) */
  const int64_t *layer_ptr;      /* n_layers + 1 offsets */
  uint32_t n_rounds;
  uint32_t reserved;
  const uint32_t *round_layers;  /* n_rounds + 1 layer offsets, [0] = 0 */
  const uint32_t *round_meas;    /* n_rounds + 1 offsets into qubits, [0] = 0 */
  const uint32_t *qubits;        /* round_meas[n_rounds] measured qubits */
  uint64_t seed, shot;           /* key of the circuit's coins */
} qs_batch_circuit;

/* Launch shape of the persistent kernel (qs_batch_autotune picks one).
 *   threads:         256, 512 or 1024 per CTA
 *   blocks_per_sm:   CTAs per SM (0 = as many as fit)
 *   words_per_block: 64-row column words per shared-memory slice in the gate phase (1 or 2)
 *   fuse_depth:      layers per shared-memory pass in the gate phase (0 = whole round)
 *   spin_limit:      bound on each grid-barrier spin (0 = default, several seconds); when it
 *                    runs out the kernel stops and qs_batch_sync returns QS_ERR_TIMEOUT */
typedef struct qs_batch_tuning {
  uint32_t threads;
  uint32_t blocks_per_sm;
  uint32_t words_per_block;
  uint32_t fuse_depth;
  uint64_t spin_limit;
} qs_batch_tuning;

typedef struct qs_batch qs_batch;

/* Device bytes of a batch's persistent-kernel part (0 if the description is
 * invalid); the simulators of the n >= 1024 circuits allocate their own. */
size_t qs_batch_required_bytes(uint32_t count, const qs_batch_circuit *circuits);

/* Validates (as qs_pack_layers; measured qubits < n; offsets in range) and
 * uploads the batch. workspace: caller device memory of >= required bytes,
 * 256-byte aligned, or NULL to let the library cudaMalloc it. Creates the
 * worker streams and the simulators of the n >= 1024 circuits. */
int qs_batch_create(uint32_t count, const qs_batch_circuit *circuits, void *cuda_stream,
                    void *workspace, size_t workspace_bytes, qs_batch **out);

int qs_batch_destroy(qs_batch *batch);

/* Runs every circuit from |0...0> through its rounds (the first round_limit
 * rounds, 0 = all): the n < 1024 circuits in one cooperative persistent
 * kernel launch on the batch's stream, the others on the worker streams.
 * Returns when all work is enqueued (the host threads wait for their streams
 * once per block of measurements); the batch's stream then waits for the
 * worker streams, so work enqueued on it afterwards follows the whole batch.
 * tuning: NULL for the default shape of the persistent kernel. */
int qs_batch_run(qs_batch *batch, const qs_batch_tuning *tuning, uint32_t round_limit);

/* Waits for the batch's stream; QS_ERR_TIMEOUT if a grid barrier ran out,
 * QS_ERR_INTERNAL if a device self-check failed. */
int qs_batch_sync(qs_batch *batch);

/* Copies the first `count` record entries (0/1 bytes) of one circuit. Syncs. */
int qs_batch_record(qs_batch *batch, uint32_t circuit, uint8_t *dst, size_t count);

/* Selected generator rows of one circuit, in the format of qs_sim_export_rows. Syncs. */
int qs_batch_export_rows(qs_batch *batch, uint32_t circuit, const uint32_t *rows, uint32_t count,
                         uint64_t *dst);

/* Times the candidate launch shapes of the persistent kernel on this batch
 * (the first round_limit rounds; 0 = all; the worker streams are idle
 * meanwhile) and returns the fastest. cache_path: NULL, or a text file
 * of "device|batch-signature|rounds threads blocks_per_sm words_per_block
 * fuse_depth" lines that is read first and appended to. Results do not depend
 * on the shape. */
int qs_batch_autotune(qs_batch *batch, uint32_t round_limit, const char *cache_path,
                      qs_batch_tuning *best);

/*
 * Pauli-frame sampling (Sec. 5, Alg. 9) of the batch's circuits after a
 * complete qs_batch_run: circuit c gets shots[c] shots (0 skips it) with frame
 * seed seeds[c] into records[c], a DEVICE pointer of [M_c][ceil(shots[c]/64)]
 * words (M_c = the circuit's measurements; bit s of word j = shot 64 j + s,
 * bits >= shots[c] are 0). The words are those qs_sim_sample gives for the same
 * circuit alone with that seed: the reference record is the circuit's batch
 * record and the frame rules are the same. The circuits of n < 1024 are sampled
 * in ONE launch on the batch's stream (a block per circuit and 64-shot word runs
 * the circuit's whole program on frames in shared memory); the others replay
 * their simulators' op logs on the worker streams, which the batch stream then
 * waits for. The paper has no batch mode; this serves many small sampling
 * requests at once. Allocates a small table on the batch's stream and waits
 * for its upload; the sampling itself is only enqueued (qs_batch_sync waits).
 * Errors: QS_ERR_ARG (NULL arrays, a NULL records[c] with shots[c] > 0,
 * shots above 2e9), QS_ERR_STATE (no complete run yet, e.g. only a round_limit
 * run or autotuning since create).
 */
int qs_batch_sample(qs_batch *batch, const uint64_t *shots, const uint64_t *seeds, uint64_t *const *records);

/* Message for the last batch error on the calling thread. */
const char *qs_batch_last_error(void);

/*
 * Window scheduling (Sec. 4.2, ScheduleWindows of Alg. 2) of an ordered list of
 * gates and measurements (type QS_MEASURE) on n qubits. Repeatedly: every gate
 * that is the first remaining operation on all its qubits forms one window of
 * parallel gates (a layer); then every measurement that has become first on its
 * qubit is emitted in ascending qubit order, each as its own window, or all as
 * one window when merge_measurements (the paper's sampling mode). Dependencies
 * on each qubit are kept; this reproduces the worked example of Sec. 4.2.
 *   out_ops:         count reordered operations
 *   out_window_ptr:  count + 1 offsets; window w = out_ops[ptr[w] .. ptr[w+1])
 *   out_window_kind: count entries, 0 = gates, 1 = measurements
 *   n_windows:       number of windows written
 * Errors: QS_ERR_ARG (unknown type, qubit >= n, two-qubit gate on one qubit);
 * message via qs_schedule_last_error().
 */
int qs_schedule_windows(uint32_t n, const qs_gate *ops, uint32_t count, int merge_measurements,
                        qs_gate *out_ops, uint32_t *out_window_ptr, uint8_t *out_window_kind,
                        uint32_t *n_windows);
const char *qs_schedule_last_error(void);

/* Number of kernel launches the sim has enqueued so far. */
uint64_t qs_sim_launch_count(const qs_sim *sim);

/* Kernel classes of qs_sim_timing (the phases of Alg. 2 and of the blocked
 * measurement): gate layers (Sec. 4.4), the layout switch between column- and
 * row-major (Sec. 4.5), the blocked measurement's symbolic pass, its pivot
 * rows with their signs and the list of rows the block changes, its apply
 * pass over the row-major tableau and its
 * per-row signs and record, measurements outside blocks (single and
 * pipelined), and frame sampling (Sec. 5). */
enum {
  QS_TIME_GATES = 0,
  QS_TIME_TRANSPOSE = 1,
  QS_TIME_BLK_SYMBOLIC = 2,
  QS_TIME_BLK_PIVOT_ROWS = 3,
  QS_TIME_BLK_APPLY = 4,
  QS_TIME_BLK_SIGNS = 5,
  QS_TIME_MEASURE_SINGLE = 6,
  QS_TIME_SAMPLE = 7,
  QS_NUM_TIME_KINDS = 8
};

/*
 * Turns CUDA-event timing of the kernel classes on (on != 0) or off and
 * clears the totals. While on, the sim records an event pair on its stream
 * around each group of launches of one class (one pair per call, layout
 * switch or block phase); the events only timestamp the stream, the kernels
 * are unchanged. Off by default. The paper has no counterpart; it times its
 * phases the same way (Sec. 6 tables).
 */
int qs_sim_set_timing(qs_sim *sim, int on);

/*
 * Waits for the stream and writes, for kind k < kinds (at most
 * QS_NUM_TIME_KINDS), the summed device milliseconds ms[k] and the number of
 * timed groups count[k] since timing was turned on. Either pointer may be
 * NULL. Errors: QS_ERR_ARG (NULL sim), QS_ERR_STATE (timing is off).
 */
int qs_sim_timing(qs_sim *sim, double *ms, uint64_t *count, uint32_t kinds);

#ifdef __cplusplus
}
#endif

#endif /* QS_GB300_API_H_ */
