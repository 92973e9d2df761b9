/*
 * hd.h -- C ABI of the GB300 (sm_103a) Huffman decoder for error-bounded lossy
 * compression codes.
 *
 * The library decodes canonical-Huffman streams of uint16 quantization codes
 * (the Lorenzo residues a cuSZ-style compressor produces) from a dense,
 * most-significant-bit-first uint32 bitstream into a uint16 array on the GPU.
 * It implements the two start-point strategies the paper (Rivera et al.,
 * "Optimizing Huffman Decoding for Error-Bounded Lossy Compression on GPUs",
 * IPDPS 2022) optimises:
 *   - gap arrays (Sec. III-C): one byte per subsequence tells each thread
 *     where its first codeword starts;
 *   - self-synchronisation (Sec. III-B, Sec. IV-A): threads start at evenly
 *     spaced positions and agree on true codeword boundaries.
 * Output offsets come from a prefix sum of per-subsequence codeword counts
 * (Sec. III-B2 step 3) and symbols are staged in shared memory before
 * coalesced stores (Sec. IV-B, Algorithm 1).
 *
 * Stream format (shared by hd_encode and every decode entry point):
 *   - bit b of the stream is bit 31 - (b mod 32) of unit floor(b / 32);
 *   - `nbits` valid bits, then zero padding to a multiple of the subsequence
 *     size S bits, then one zero guard unit:
 *     nwords = ceil(nbits / S) * S / 32 + 1 (S a multiple of 32);
 *   - codewords are canonical (RFC 1951 Sec. 3.2.2 assignment) for the code
 *     lengths `lengths[alphabet]` (0 = symbol absent, at most 32 bits);
 *   - gap array (optional): gap[i] = (first codeword boundary at or after
 *     bit i*S) - i*S, one uint8 per subsequence, in [0, 31].  The boundaries
 *     are the codeword starts and the stream end.  The paper's example
 *     [0, 0, -2, -1] (Sec. III-C) uses the signed offset to the codeword that
 *     straddles the boundary; the two conventions differ by that codeword's
 *     length.
 *
 * Ownership: every pointer stays owned by the caller.  Device pointers must
 * stay valid until the work queued on the given stream has finished.
 * Errors are returned as negative status codes; no exception crosses the ABI.
 * A context may be used from several host threads (calls are serialised by
 * an internal lock) but decodes queued on one context must not overlap on the
 * device: use one context per concurrently running stream.
 */
#ifndef HD_H
#define HD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HD_OK 0
#define HD_PENDING 1        /* serve: request not finished yet */
#define HD_ERR_ARG (-1)     /* invalid argument, size or alignment */
#define HD_ERR_CAPACITY (-2)/* output buffer too small (required sizes reported) */
#define HD_ERR_SYMBOL (-3)  /* input symbol outside the alphabet or without code */
#define HD_ERR_CORRUPT (-4) /* stream is no valid encoding of n symbols */
#define HD_ERR_NOSYNC (-5)  /* self-synchronisation did not converge in its cap */
#define HD_ERR_TIMEOUT (-6) /* a device-side wait gave up (hd_decode_static) */
#define HD_ERR_CUDA (-7)    /* a CUDA runtime call failed */
#define HD_ERR_NOMEM (-8)   /* host or device allocation failed / over budget */
#define HD_ERR_BUSY (-9)    /* serve: queue full or server stopped */

/* ---- host-side codebook construction and encoding (test-input generation) */

typedef struct hd_stream_info {
  uint64_t nbits;  /* valid bits in the stream */
  uint64_t nwords; /* uint32 units including padding and the guard unit */
  uint64_t nsub;   /* subsequences = gap entries = ceil(nbits / S) */
} hd_stream_info;

/* Code lengths of an optimal prefix code for the histogram of codes[0..n)
 * (Huffman's construction, Sec. II-B), limited to max_len bits with
 * package-merge when the Huffman tree is deeper.  A single used symbol gets
 * length 1.  Host memory.  Errors: HD_ERR_ARG if alphabet is not in [2, 65536]
 * or max_len not in [1, 32] or more than 2^max_len symbols are used;
 * HD_ERR_SYMBOL if a code is >= alphabet. */
int hd_build_codebook(const uint16_t* codes, uint64_t n, uint32_t alphabet, uint32_t max_len,
                      uint8_t* lengths_out);

/* Canonical-Huffman encodes codes[0..n) into the stream format above, with
 * subsequences of subseq_bits (64, 128 or 256) and, when gap_out is not NULL,
 * the gap array.  Host memory.  `info` always receives the required sizes.
 * Errors: HD_ERR_CAPACITY if words_cap < info->nwords or (gap_out != NULL and)
 * gap_cap < info->nsub; HD_ERR_SYMBOL for a symbol with length 0 or outside
 * the alphabet; HD_ERR_ARG for an invalid length table (Kraft sum > 1). */
int hd_encode(const uint16_t* codes, uint64_t n, const uint8_t* lengths, uint32_t alphabet,
              uint32_t subseq_bits, uint32_t* words_out, uint64_t words_cap, uint8_t* gap_out,
              uint64_t gap_cap, hd_stream_info* info);

/* Code lengths of an optimal prefix code for the symbol counts freq[alphabet]
 * (as hd_build_codebook, from counts instead of symbols, e.g. those of
 * hd_histogram_device).  Host memory.  Errors as hd_build_codebook. */
int hd_build_codebook_freq(const uint64_t* freq, uint32_t alphabet, uint32_t max_len,
                           uint8_t* lengths_out);

/* ---- device context ---------------------------------------------------- */

typedef struct hd_ctx hd_ctx;

/* Creates a context bound to CUDA device `device`.  The context owns its
 * device workspace (decode tables, per-subsequence codeword counts and
 * starts, per-tile totals, error words), which grows on demand with
 * cudaMalloc outside of any decode call's device work. */
int hd_ctx_create(int device, hd_ctx** out);
int hd_ctx_destroy(hd_ctx* ctx);

/* One encoded field.  All pointers are device pointers for hd_decode and
 * hd_decode_batch, host pointers for hd_decode_host. */
typedef struct hd_field {
  const uint32_t* words;    /* stream, nwords units, 16-byte aligned */
  uint64_t nwords;          /* must be >= ceil(nbits / S) * S / 32 + 1 */
  uint64_t nbits;           /* valid bits */
  const uint8_t* gap;       /* gap array or NULL (=> self-synchronisation) */
  uint32_t subseq_bits;     /* S the stream/gap array was written with: 64, 128, 256 */
  const uint8_t* lengths;   /* code lengths [alphabet] */
  uint32_t alphabet;        /* 2 .. 65536 */
  uint64_t n;               /* number of symbols encoded in the stream */
} hd_field;

/* Launch shape (0 = library default / autotuned choice). */
typedef struct hd_config {
  uint32_t subseq_bits; /* decoder subsequence bits.  Gap-array decode: a multiple
                           of the field's S, <= 512 (0 = max(256, S));
                           self-synchronisation: 64, 128 or 256 (512 acts as
                           256; 0 = 256); hd_sync_points always uses the
                           field's S */
  uint32_t threads;     /* threads per block: 128, 256, 512 (two phases: one
                           subsequence per thread, a tile per block); one pass
                           also 768 and 1024 (a tile per warp) */
  uint32_t window;      /* shared-memory output window in symbols (Alg. 1 buffer);
                           0 = sized from the field's mean code length */
  uint32_t lut_bits;    /* first-level decode-table index bits, 8 .. 15 (0 = 13
                           for alphabets up to 4096, whose tables have 16-bit
                           entries, else 12); a shape whose tables do not fit
                           shared memory fails with HD_ERR_ARG */
  uint32_t cr_classes;  /* gap-array hd_decode only: 0 = one output window for
                           all tiles; 2 .. 32 = per-tile compression-ratio
                           classes (Sec. IV-C, Algorithm 2): after counting,
                           tiles are sorted on the GPU into classes by their
                           codeword count, the class sizes are read back, and
                           one decode-and-write launch per class runs with a
                           window sized for that class's largest tile (capped
                           by shared memory) */
  uint32_t decoder;     /* gap-array decodes: 0 = automatic (one pass for a single
                           field, two phases for batches, CR classes and
                           decode + reconstruction), 1 = two phases (count
                           kernel, tile scan, decode-and-write kernel), 2 = one
                           pass: each warp decodes 32 subsequences once into
                           shared memory, takes its output index from a
                           look-back over the tiles before it and writes
                           through its window (single fields only) */
} hd_config;

/* Sets the launch shape used by later decodes on this context (NULL resets to
 * defaults).  HD_ERR_ARG for values outside the ranges above.  hd_get_config
 * reports the configured values, with the shape of the last decode in place
 * of those left at 0. */
int hd_set_config(hd_ctx* ctx, const hd_config* cfg);
int hd_get_config(hd_ctx* ctx, hd_config* cfg);

/* Decodes field `f` into d_out[0 .. f->n) on `stream` (a cudaStream_t, NULL =
 * legacy default stream).  Asynchronous: argument errors are returned
 * immediately; stream errors are recorded on the device and returned by
 * hd_status.  With a gap array the start of every subsequence is read from
 * it; without one it is found by self-synchronisation.  d_out must be 2-byte
 * aligned and hold f->n elements; nothing outside it is written, even for a
 * corrupt stream. */
int hd_decode(hd_ctx* ctx, const hd_field* f, uint16_t* d_out, void* stream);

/* Waits for `stream` and returns the status of the last hd_decode /
 * hd_sync_points / hd_decode_batch queued on this context: HD_OK,
 * HD_ERR_CORRUPT (stream, gap array or n inconsistent), HD_ERR_ARG (length
 * table with Kraft sum > 1 or a length > 32), HD_ERR_NOSYNC or HD_ERR_CUDA. */
int hd_status(hd_ctx* ctx, void* stream);

/* Self-synchronisation only (Sec. III-B2 steps 1-2): computes the gap array
 * gap_out[0 .. ceil(nbits/S)) of field `f` (whose `gap` is ignored) from the
 * bitstream, with S = f->subseq_bits.  Device pointers, asynchronous, status
 * via hd_status. */
int hd_sync_points(hd_ctx* ctx, const hd_field* f, uint8_t* gap_out, void* stream);

/* Inspection of the per-prefix decode tables the kernels build from a code-
 * length table (Sec. II-B canonical codes; the first-level tables of a1), for
 * tests and tools.  Builds the tables of `lengths` (a DEVICE pointer,
 * `alphabet` entries, 2 .. 4096) with K first-level bits (8 .. 15) in a
 * temporary device buffer of its own, exactly as a decode on this context
 * builds them, and copies the 2^K entries of each requested table to the host
 * (any pointer may be NULL):
 *   lut16[p]: for a code of at most K bits at prefix p, its length << 12 |
 *             its symbol; else 0 << 12 | the smallest length under p, with
 *             bit 11 (0x800) set when p holds codes of several lengths;
 *   len8[p]:  the code length when every code under p has one length, else
 *             0x80 | the smallest length (33: no code);
 *   run8[p]:  m << 4 | b: the m (1 .. 7) codes that lie wholly within the K
 *             bits of p, decoded one after another from the first, take b
 *             bits; 0 when the first code is longer than K bits;
 *   pair[p]:  the two-code entry of the decode-and-write kernel: m (the codes
 *             of p's K bits it resolves, up to two) << 30; m = 2 (alphabets
 *             up to 1024): first length << 26 | second length << 22 | second
 *             symbol << 10 | first symbol; m = 1: first length << 26 | its
 *             symbol; m = 0: as lut16 for a longer first code.
 * Synchronous on `stream`.  HD_ERR_ARG for bad arguments, HD_ERR_CORRUPT for a
 * length table that is no prefix code, HD_ERR_CUDA when an allocation or copy
 * fails. */
int hd_inspect_tables(hd_ctx* ctx, const uint8_t* lengths, uint32_t alphabet, uint32_t K,
                      uint16_t* lut16, uint8_t* len8, uint8_t* run8, uint32_t* pair,
                      void* stream);

/* Decodes nf independent fields of any sizes (device pointers, own codebooks;
 * Sec. III-C / III-B per field) with one CUDA graph launch for all gap-array
 * fields and one for all self-synchronising fields; d_outs[i] receives field
 * i.  The persistent kernels spread the tiles of all fields over the GPU and
 * read the batch's sizes from device memory, so a graph captured once per
 * (strategy, launch shape, power-of-two capacity class) is replayed for every
 * later batch that fits it.  The launch shape is the context's configuration
 * when one is set, else the shape hd_autotune chose for the batch's class,
 * else the defaults.  Asynchronous except that, when both strategies occur,
 * the call waits for the first group before queuing the second.  Per-field
 * status via hd_batch_status. */
int hd_decode_batch(hd_ctx* ctx, const hd_field* fs, uint32_t nf, uint16_t* const* d_outs,
                    void* stream);
/* Waits for `stream`; status[i] = status of field i of the last batch. Returns
 * the first non-OK status or HD_OK. */
int hd_batch_status(hd_ctx* ctx, int32_t* status, uint32_t nf, void* stream);

/* Autotuner (launch-configuration choice; the paper tunes the shared-memory
 * buffer per sequence online, Sec. IV-C, Algorithm 2): decodes the batch with
 * every candidate shape -- decoder subsequence bits {64, 128, 256, 512} (a
 * multiple of the largest stream S for gap arrays, at most 256 for
 * self-synchronisation) x threads {128, 256, 512} x first-level table bits
 * {11, 12, 13, 14}, window sized from the mean code length -- timing three
 * replays of each with CUDA events, and keeps the fastest shape that decodes
 * every field without error.  The choice is stored in the context per batch
 * class (strategy, mean code length in quarter bits, log2 of the symbol
 * count, largest stream S) and used by later hd_decode_batch calls of that
 * class, and by hd_decode / hd_decode_host calls of a single field of that
 * class, while the context's configuration is all zero.  `best` (may be NULL)
 * receives the shape chosen for the first strategy group.  Synchronous; the
 * outputs hold the batch's symbols afterwards.  HD_ERR_CORRUPT if no
 * candidate decodes the batch cleanly. */
int hd_autotune(hd_ctx* ctx, const hd_field* fs, uint32_t nf, uint16_t* const* d_outs,
                void* stream, hd_config* best);

/* Keeps the autotuner's choices across processes: hd_autotune_save writes
 * every batch class this context has tuned, with the device's name, to the
 * text file `path` (replacing it); hd_autotune_load reads such a file and
 * takes the entries of the same device name into this context, as if
 * hd_autotune had chosen them (*loaded = their number).  HD_ERR_ARG for a
 * file that cannot be opened or is not such a file (nothing is loaded then). */
int hd_autotune_save(hd_ctx* ctx, const char* path);
int hd_autotune_load(hd_ctx* ctx, const char* path, uint32_t* loaded);

/* Graph statistics of a context: graphs captured since creation and graphs
 * currently cached. */
int hd_graph_stats(hd_ctx* ctx, uint64_t* captures, uint32_t* cached);

/* Host-buffer decode: `f` holds HOST pointers (pinned memory is fastest),
 * host_out receives f->n symbols.  Copies the stream, gap array and lengths
 * to context-owned device buffers, decodes and copies the symbols back;
 * returns when done with the decode status.  Large gap-array fields run as a
 * pipeline (the transfers belong to the paper's end-to-end comparison,
 * Sec. V): the stream goes to the device in chunks of whole tiles on one copy
 * stream, each chunk is counted, scanned and decoded on `stream` once its bits
 * have arrived, and its symbols return on a second copy stream once written,
 * so both transfer directions and the kernels overlap.  Other fields are
 * copied, decoded and copied back in sequence on `stream`. */
int hd_decode_host(hd_ctx* ctx, const hd_field* f, uint16_t* host_out, void* stream);

/* Allocation-free gap-array decode.  Some callers cannot call cudaMalloc
 * when they decode: real-time loops that cannot afford the device-wide
 * synchronisation cudaMalloc may imply, and plugins or libraries running
 * inside a host framework whose own allocator has already reserved the device
 * memory.  This entry point needs no context and allocates nothing.  Its
 * scratch (control words, look-back states and the decode table) is one fixed
 * 1 MiB array in device memory that every GPU which loads the library holds
 * until the process exits.  Arguments are as for hd_decode (device pointers);
 * the field must carry a gap array (NULL gap -> HD_ERR_ARG).  A field whose
 * scratch would not fit in the 1 MiB -- more than about 128,000 tiles of 256
 * subsequences, i.e. a stream beyond roughly 500 MB at S = 128 with a
 * 1024-symbol alphabet -- is rejected with HD_ERR_CAPACITY before any GPU
 * work.  The first
 * call on each device does a one-time set-up (it looks up the array's device
 * address with that device current); make that first call before any stream
 * capture.  That address is kept for the life of the process: after a
 * cudaDeviceReset (or anything else that recreates the device's primary
 * context) it would be stale, so such a reset is not supported in a process
 * that has called this entry point.  All calls on a device share the one array, which keeps the last
 * call's contents: each call clears the parts that must start at zero, but
 * calls whose GPU work overlaps (e.g. issued on two streams at once) race on
 * it and give wrong results.  The call waits for its work on `stream` and
 * returns the decode status (HD_OK, HD_ERR_CORRUPT, HD_ERR_TIMEOUT, ...).
 * The paper has no counterpart to this entry point. */
int hd_decode_static(const hd_field* f, uint16_t* d_out, void* stream);

/* ---- serving loop ------------------------------------------------------- */

/* A server decodes requests against resident fields: each request names a
 * registered field and receives a fresh device copy of its symbols.  One
 * worker thread keeps up to `slots` batches in flight, each on its own stream
 * with its own decode context, so requests that arrive while others are on
 * the GPU are admitted as soon as a slot and budget memory are free and their
 * work overlaps the running batches (continuous batching).  Admission is
 * first come, first served: the oldest pending requests whose outputs fit the
 * budget (up to max_batch) form the next batch, which is decoded by one
 * hd_decode_batch call.  The paper has no counterpart to the server; each
 * batch runs the paper's decoders (Sec. III-B/III-C, Algorithm 1). */
typedef struct hd_server hd_server;

typedef struct hd_serve_config {
  uint64_t budget_bytes; /* device memory for request outputs (one allocation at
                            creation; a request is admitted only when its
                            2*n-byte output fits what is not yet released) */
  uint32_t slots;        /* batches in flight at once, 1 .. 8 */
  uint32_t max_batch;    /* requests per batch, 1 .. 4096 */
  uint32_t queue_cap;    /* pending requests before submit returns HD_ERR_BUSY
                            (0 = 2^20) */
  uint32_t direct;       /* 1: one hd_decode launch per request instead of a
                            batch (requires max_batch == 1; the baseline the
                            batched server is compared with) */
  uint32_t watchdog_us;  /* limit on a batch's time on the GPU, microseconds
                            (0 = 10 s).  Past it, the batch's requests complete
                            with status HD_ERR_TIMEOUT and no output; the slot
                            and their output memory stay held (the GPU may
                            still write there) until the work really ends */
} hd_serve_config;

typedef struct hd_result {
  int32_t status;        /* decode status of the request */
  const uint16_t* d_out; /* device pointer to its n symbols, valid until release */
  uint64_t n;
  double queue_us;       /* submission to launch */
  double latency_us;     /* submission to observed completion */
} hd_result;

typedef struct hd_serve_stats_t {
  uint64_t submitted, completed, batches, pending, in_flight;
  uint64_t budget_bytes, used_bytes, peak_bytes;
  uint64_t timed_out_batches; /* batches past the watchdog, still on the GPU */
  uint64_t retired_batches;   /* timed-out batches that ended later */
} hd_serve_stats_t;

/* Creates a server on `device` (`shape` may be NULL: default or autotuned
 * launch shapes; else the shape every slot uses).  HD_ERR_ARG for a config
 * outside the ranges above, HD_ERR_NOMEM if the budget cannot be allocated. */
int hd_serve_create(int device, const hd_serve_config* cfg, const hd_config* shape,
                    hd_server** out);
/* Drops pending requests (their status becomes HD_ERR_BUSY), waits for the
 * batches in flight, frees everything (outputs included). */
int hd_serve_destroy(hd_server* srv);
/* Registers a resident field (device pointers, as for hd_decode; they stay
 * owned by the caller and must outlive the server).  Returns its id. */
int hd_serve_register(hd_server* srv, const hd_field* f, uint32_t* field_id);
/* Queues a decode of field `field_id`; returns at once with a ticket.
 * HD_ERR_BUSY if the queue is full, HD_ERR_NOMEM if the output can never fit
 * the budget. */
int hd_serve_submit(hd_server* srv, uint32_t field_id, uint64_t* ticket);
/* HD_PENDING while the request is queued or on the GPU; HD_OK with *res
 * filled once it completed (res->status holds its decode status). */
int hd_serve_poll(hd_server* srv, uint64_t ticket, hd_result* res);
/* Returns a completed request's output memory to the budget and forgets the
 * ticket (HD_ERR_BUSY if it has not completed). */
int hd_serve_release(hd_server* srv, uint64_t ticket);
/* Hands out up to `cap` tickets of requests that completed since the last
 * call (in completion order); *count receives how many. */
int hd_serve_completed(hd_server* srv, uint64_t* tickets, uint32_t cap, uint32_t* count);
/* Waits until no request is pending or in flight.  Requests wait for budget
 * memory, so outputs must be released meanwhile if the budget is short. */
int hd_serve_drain(hd_server* srv);
int hd_serve_stats(hd_server* srv, hd_serve_stats_t* out);

/* ---- Reconstruction (the step after the decoder) ------------------------ */

/* cuSZ's Lorenzo reconstruction, the second half of the end-to-end
 * decompression the paper measures (Sec. V-B2; the paper cites cuSZ for it
 * and does not define it).  Reading: first-order Lorenzo prediction on
 * prequantized integers, zero outside the domain.  A code c in [1, 2R)
 * stands for the residue d = c - R; code 0 marks an outlier whose residue is
 * stored aside.  The prequantized value q is the inclusive prefix sum of d
 * along every axis, and the output value is float32(q) * float32(2 eb) (each
 * conversion rounded to nearest even).  q must stay within int32. */
typedef struct hd_lorenzo {
  uint32_t ndim;           /* 1, 2 or 3 */
  uint32_t radius;         /* R, 1 .. 32768 */
  uint64_t dims[3];        /* extents, dims[0] varying fastest; entries >= ndim ignored.
                              2D/3D: dims[0] <= 49152 */
  double eb;               /* absolute error bound (finite, >= 0) */
  const uint64_t* out_idx; /* device: ascending positions whose code is 0 [n_out] */
  const int32_t* out_val;  /* device: their residues [n_out] */
  uint64_t n_out;
  uint32_t chunk_slices;   /* band path, 3D: slices reconstructed per group, whose
                              int32 intermediate may stay in L2 (0 = about 32 MB
                              of it) */
  uint32_t band_rows;      /* band path: rows per band, 1 .. 64 (0 = 8 for rows
                              up to 1024 codes, else as many as 64 KB of shared
                              memory holds, at most 32) */
  uint32_t separate;       /* hd_decompress_device, 1D gap-array fields: 1 = decode
                              into codes, then reconstruct; 0 = fused (values
                              straight from the decoder) */
  uint32_t pad;
} hd_lorenzo;

/* Reconstructs dims[0]*..*dims[ndim-1] float32 values into d_out (device,
 * 16-byte aligned) from the codes d_codes (device, 16-byte aligned).
 * 1D: residue sums of tiles of 8192 codes, their scan, and a pass that
 * rescans each tile from its prefix.
 * 3D with rows up to 1024 codes and at least two slices per SM (and
 * chunk_slices = band_rows = 0), the slice path: one block per slice for the
 * x and y prefixes (int32 written into d_out), then a z kernel that writes
 * the floats in place.
 * Otherwise the band path: per group of slices a band kernel (a warp per
 * band of rows in registers, or a block per band in shared memory for longer
 * rows), a band-carry scan and the z kernel with the carries.
 * Queued on `stream`; hd_status reports HD_ERR_CORRUPT for a code 0 the
 * outlier list lacks (its residue is taken as 0).  HD_ERR_ARG for invalid
 * parameters or alignment. */
int hd_reconstruct_device(hd_ctx* ctx, const uint16_t* d_codes, const hd_lorenzo* L,
                          float* d_out, void* stream);

/* Decompression of f (device field, f->n = the grid size) into float32
 * values d_out (device, 16-byte aligned).  1D gap-array fields (unless
 * L->separate): fused -- the count kernel also sums each tile's residues,
 * the tile scan scans them, a tile kernel adds the outliers' corrections and
 * the decode-and-write kernel turns each output window into values (a block
 * scan from the tile's q) instead of storing codes; no codes reach HBM.
 * Otherwise hd_decode into a context-owned code buffer, then
 * hd_reconstruct_device.  One status for both through hd_status. */
int hd_decompress_device(hd_ctx* ctx, const hd_field* f, const hd_lorenzo* L, float* d_out,
                         void* stream);

/* ---- GPU encoding (the step before the decoder) ------------------------- */

/* Symbol counts of d_codes[0 .. n) (device) into freq_out[alphabet] (host).
 * Synchronous.  HD_ERR_SYMBOL if a code is >= alphabet. */
int hd_histogram_device(hd_ctx* ctx, const uint16_t* d_codes, uint64_t n, uint32_t alphabet,
                        uint64_t* freq_out, void* stream);

/* GPU counterpart of hd_encode, bit-identical to it: canonical-Huffman
 * encodes d_codes[0 .. n) (device, 2-byte aligned) with the code lengths
 * `lengths` (HOST, [alphabet]) into d_words (device, 4-byte aligned) in the
 * stream format above and, when d_gap is not NULL, writes the gap array of
 * subseq_bits-bit subsequences (Sec. III-C) into d_gap.  Symbol tiles are
 * sized by a per-tile bit count and a scan, then every codeword is OR-ed into
 * place in shared memory and the gap entry of each subsequence is written by
 * the thread placing its first codeword.  Synchronous (the stream length is
 * needed to check capacities); `info` always receives the sizes.  Errors as
 * hd_encode (HD_ERR_CAPACITY, HD_ERR_SYMBOL, HD_ERR_ARG), HD_ERR_CUDA. */
int hd_encode_device(hd_ctx* ctx, const uint16_t* d_codes, uint64_t n, const uint8_t* lengths,
                     uint32_t alphabet, uint32_t subseq_bits, uint32_t* d_words,
                     uint64_t words_cap, uint8_t* d_gap, uint64_t gap_cap, hd_stream_info* info,
                     void* stream);

/* Limit on each device-side wait of the one-pass decoder (a tile waiting in
 * its look-back for the counts of the tiles before it), in SM clock cycles;
 * 0 restores the default of about 2 s.  A wait that reaches the limit gives
 * up, every later wait of that decode returns at once, the decode still
 * writes nothing outside its output, and hd_status reports HD_ERR_TIMEOUT;
 * the context stays usable.  A very short limit makes waits give up on
 * purpose, which is how failure detection is tested without hanging a GPU. */
int hd_set_wait_limit(hd_ctx* ctx, uint64_t cycles);

/* Kernel timing: when enabled, the context records CUDA events around every
 * main decode kernel it launches.  hd_kernel_time waits for them and returns
 * the summed device time in milliseconds and the launch count, then clears. */
int hd_profile(hd_ctx* ctx, int enable);
int hd_kernel_time(hd_ctx* ctx, double* ms, uint64_t* launches);

/* Per-phase device time of the single-field decodes queued on this context
 * while profiling (hd_profile) since the last call, in milliseconds summed over
 * those decodes, mirroring the phases the paper times (Sec. V-B):
 *   ms[0] synchronisation: finding the subsequence starts without a gap array
 *         (Sec. III-B2 steps 1-2, the self-synchronising kernels);
 *   ms[1] counting the codewords of every subsequence (gap-array count kernel);
 *   ms[2] output indices: the prefix sum over tiles (Sec. III-B2 step 3);
 *   ms[3] decode and write (Algorithm 1); for the one-pass decoder, whose one
 *         kernel counts, takes its indices and writes, the whole pass.
 * With profiling on, the two-phase kernels are queued one phase at a time with
 * an event between phases.  *decodes receives the number of decodes summed.
 * Waits for the events and clears them.  Batches (graph launches) are not
 * split into phases. */
int hd_phase_times(hd_ctx* ctx, double* ms, uint64_t* decodes);

/* Number of kernel launches the context has issued since creation. */
uint64_t hd_launch_count(hd_ctx* ctx);

/* Library version string. */
const char* hd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HD_H */
