/*
 * recoil.h -- C-ABI of the B300 Recoil decoder.
 *
 * Recoil (Lin et al., "Recoil: Parallel rANS Decoding with Decoder-Adaptive
 * Scalability", ICPP 2023) encodes data once as ONE 32-way interleaved rANS
 * bitstream (Sec. 2.2) and records split metadata: for a split word, each
 * coder's state right after its last renormalisation at or before that word
 * (bounded by L, Lemma 3.1) and the index of the last symbol it coded
 * (Sec. 3.1, 4.1). Decoders start at any recorded split, synchronise, decode,
 * and cross into the previous split's synchronisation section (Sec. 4.1.1-4.1.3).
 * Splits are combined by dropping metadata entries (Sec. 3.3, 4.2).
 *
 * Fixed parameters (Sec. 4.4, Table 3): 32-bit states, 8- or 16-bit symbols,
 * L = 2^16, 16-bit renormalisation words, n <= 16 quantisation bits, W = 32.
 *
 * Conventions
 *   - Every function returns RECOIL_OK (0) or a negative RECOIL_E* code; the
 *     message of the last failure on the calling thread is recoil_last_error().
 *   - Host objects (recoil_stream, recoil_plan) are owned by the library and
 *     released with recoil_free / recoil_plan_free.
 *   - Device memory (workspaces, outputs) is owned by the caller: plain device
 *     pointers, e.g. from torch tensors' data_ptr(). The library never
 *     allocates device memory.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Decoding is asynchronous on it.
 *   - Symbols are little-endian uint8 or uint16 arrays of n_syms elements.
 *   - Nothing here is thread-safe on the same object; distinct objects may be
 *     used from distinct threads.
 */
#ifndef RECOIL_H
#define RECOIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RECOIL_W 32        /* interleaved coders per stream (Sec. 4.4, Table 3) */
#define RECOIL_LOG2_L 16   /* renormalisation lower bound L = 2^16 (Table 3) */
#define RECOIL_B 16        /* bits per renormalisation word b (Table 3) */

#define RECOIL_OK 0
#define RECOIL_EINVAL (-1)     /* bad argument: null pointer, n outside [1,16], alphabet too large, ... */
#define RECOIL_ECORRUPT (-2)   /* metadata failed validation, or a kernel found an inconsistent stream */
#define RECOIL_ENOMEM (-3)     /* host allocation failed, or a caller buffer is too small */
#define RECOIL_ECUDA (-4)      /* a CUDA runtime call failed (message has the CUDA error) */
#define RECOIL_ETIMEOUT (-5)   /* a bounded wait expired (serving runtime) */

/* Split rules: the expected symbols per split T in the heuristic of Def. 4.1 / Eq. 7. */
#define RECOIL_SPLIT_REMAINING 0u  /* T = ceil((N - lo) / (M - k)) over the symbols left (default) */
#define RECOIL_SPLIT_EQ7 1u        /* T = ceil(N / M) for every split, as Def. 4.1 prints it */

/* Coding parameters of a stream. n_bits in [1,16] (b = 16 >= n, Sec. 4.4);
 * sym_bytes 1 (uint8 symbols) or 2 (uint16 symbols); split_rule one of
 * RECOIL_SPLIT_* (used where splits are placed; 0 = the default); reserved 0. */
typedef struct {
  uint32_t n_bits;
  uint32_t sym_bytes;
  uint32_t split_rule;
  uint32_t reserved;
} recoil_params;

typedef struct recoil_stream recoil_stream;   /* opaque host object */

typedef struct {
  uint64_t n_syms;            /* N */
  uint64_t n_words;           /* 16-bit words in the bitstream */
  uint32_t n_entries;         /* split entries, including the final-state entry */
  uint32_t n_bits;
  uint32_t sym_bytes;
  uint32_t alphabet;          /* symbols of the (each) frequency table */
  uint64_t bitstream_bytes;   /* 2 * n_words + 4 * W (final states) */
  uint64_t metadata_bytes;    /* unpacked split metadata: (8 + 2W + 4W) bytes per regular entry */
  uint64_t max_sync;          /* largest synchronisation section, in symbols (Sec. 4.1) */
  uint32_t n_tables;          /* adaptive model: PDF rows (0: one static PDF) */
  uint32_t reserved;
} recoil_info;

/*
 * Encode n_syms symbols as one interleaved rANS stream (Eqs. 1 and 3, Sec. 2.2)
 * and place split entries by the heuristic of Def. 4.1 / Eq. 7: for each split
 * in turn, the usable word minimising H = |t - T| + |t - t_s - T| (t: symbols
 * since the previous split point including this split's synchronisation
 * section, t_s: that section's symbols; ties to the smaller word).
 * params->split_rule picks T: RECOIL_SPLIT_EQ7 takes the printed
 * T = ceil(N / M) for every split; RECOIL_SPLIT_REMAINING (default) takes
 * T = ceil((N - lo) / (M - k)) over the symbols left, since with the printed T
 * every split falls short of T by about half its synchronisation section and
 * the shortfall collects in the final split (on 1 GiB of Zipf bytes at 65536
 * splits: ~3.8 M symbols in the final split instead of ~16 K).
 *   syms        host array of n_syms symbols (uint8 or uint16 per params->sym_bytes)
 *   params      n_bits, sym_bytes and split_rule
 *   max_splits  splits M the decoder may use at most, counting the final-state
 *               entry; the heuristic yields at most M (fewer on short inputs)
 *   out         receives a new stream (free with recoil_free)
 * The static quantised PDF comes from the symbol counts (Sec. 5.1): present
 * symbols get f = max(1, round_half_even(c 2^n / N)), then +-1 corrections
 * until the sum is 2^n. Errors: RECOIL_EINVAL (null, n outside [1,16],
 * sym_bytes not 1/2, an unknown split_rule, more distinct symbols than 2^n,
 * n_syms >= 2^31),
 * RECOIL_ENOMEM. The encoder is serial by design (Sec. 6).
 */
int recoil_encode_with_splits(const void* syms, uint64_t n_syms, const recoil_params* params,
                              uint32_t max_splits, recoil_stream** out);

/*
 * As recoil_encode_with_splits, with the quantised PDF given instead of
 * counted: freq[alphabet] sums to 2^n and is positive for every symbol that
 * occurs (e.g. one static model shared by many streams, or by the partitions
 * of the conventional scheme the paper compares with, Sec. 2.3).
 * Errors: as above, and EINVAL for a table that is missing, does not sum to
 * 2^n, or gives an occurring symbol no probability.
 */
int recoil_encode_with_table(const void* syms, uint64_t n_syms, const recoil_params* params, const uint32_t* freq,
                             uint32_t alphabet, uint32_t max_splits, recoil_stream** out);

/*
 * Combine splits (Sec. 3.3, 4.2): a new stream with min(target_splits, K)
 * entries, keeping entries ceil((k+1) K / M') - 1 of the K entries of `in`
 * (the final-state entry always stays). The bitstream is shared, not copied;
 * `in` is untouched and may be freed independently. O(M' W). Errors: EINVAL.
 */
int recoil_combine_splits(const recoil_stream* in, uint32_t target_splits, recoil_stream** out);

/*
 * Adaptive coding (Sec. 3.1): the PDF of every coding step is chosen by the
 * symbol index, as in hyperprior image codecs. Symbol i is coded with row
 * table_index[i] of a set of quantised PDFs; the decoder reads the same table
 * numbers (the codec derives them before entropy decoding), so the stream
 * keeps a copy of them and the decoder tables hold every row.
 *   freq         n_tables * alphabet frequencies, row t = PDF t over the
 *                alphabet; every row sums to 2^n and gives every symbol a
 *                frequency >= 1 (a hyperprior codec's discretised densities
 *                do); so 2 <= alphabet <= 2^n
 *   n_tables     rows, 1..256; table_index holds n_syms bytes, each < n_tables
 *   alphabet     <= 4096 (256 for 8-bit symbols); the n_tables CDF rows must
 *                fit in shared memory with the decoder rings
 *                (n_tables * (alphabet + 1) * 2 bytes, rounded up, <= ~160 KiB);
 *                a plan adds a bucket guide per row where room is left
 * Split placement, combining and plans work as for static streams; adaptive
 * streams decode with 4, 8, 16 or 32 warps per CTA, are not serialised
 * (recoil_serialize) and not taken by recoil_decode_noalloc.
 * Errors: EINVAL (bad parameters, a row that does not sum to 2^n or has a zero,
 * a table number or symbol out of range), ENOMEM.
 */
int recoil_encode_adaptive(const void* syms, uint64_t n_syms, const recoil_params* params, const uint32_t* freq,
                           uint32_t n_tables, uint32_t alphabet, const uint8_t* table_index, uint32_t max_splits,
                           recoil_stream** out);

/* Sizes and counts of a stream. Errors: EINVAL. */
int recoil_stream_info(const recoil_stream* s, recoil_info* out);

/*
 * Copy a stream's parts out (any pointer may be NULL to skip it):
 *   freq[alphabet] (adaptive: [n_tables * alphabet]), words[n_words], final_states[W],
 *   entry_word[R], entry_index[R*W] (recorded symbol index per coder),
 *   entry_state[R*W] (16-bit states), R = n_entries - 1 regular entries.
 */
int recoil_stream_export(const recoil_stream* s, uint32_t* freq, uint16_t* words,
                         uint32_t* final_states, uint64_t* entry_word, uint64_t* entry_index,
                         uint16_t* entry_state);

/*
 * Build a stream from parts made elsewhere (e.g. another encoder). Validates
 * the metadata (Sec. 4.1): frequencies sum to 2^n, words strictly increase,
 * every recorded index is congruent to its coder modulo W and below n_syms,
 * states are < L (Lemma 3.1), each entry's smallest index does not decrease,
 * and the top coder's join lies within the stream. Errors: EINVAL, ECORRUPT.
 */
int recoil_stream_import(const recoil_params* params, uint64_t n_syms, uint32_t alphabet,
                         const uint32_t* freq, const uint16_t* words, uint64_t n_words,
                         const uint32_t* final_states, uint32_t n_regular,
                         const uint64_t* entry_word, const uint64_t* entry_index,
                         const uint16_t* entry_state, recoil_stream** out);

/* Move the stream's words to page-locked host memory (faster host->device
 * copies). Needs a CUDA driver. Errors: ECUDA. */
int recoil_stream_pin(recoil_stream* s);

/*
 * Serialised form of a stream: what a content server stores and sends
 * (Sec. 3.3). Little-endian container: "RCL1", n_bits (u8), sym_bytes (u8),
 * two zero bytes, alphabet (u32), the quantised PDF (u32 each), the W final
 * states (u32 each), the word count (u64), the words (u16 each), the length of
 * the metadata section in bytes (u64), then the split metadata packed as in
 * Sec. 4.3:
 *   - header: M = splits counting the final-state one (32 bits), words B (64),
 *     symbols N (64);
 *   - the split words q_i, i = 1..M-1, as differences from i*ceil(B/M), and
 *     the anchors (largest group ID of a split point, group ID = recorded
 *     index / W + 1, Table 2) as differences from i*ceil(ceil(N/W)/M): two
 *     signed series (Table 1);
 *   - per split point its W states as-is (16 bits each, Lemma 3.1) and the
 *     series of anchor minus each coder's group ID (unsigned, Table 2).
 * A series is (w-1) in a 4-bit (unsigned) or 5-bit (signed) field, then each
 * value in w bits, a signed value after a sign bit; w = the bit length of the
 * largest magnitude, 1 when all are zero. Bits go most significant first; the
 * section is padded with zero bits to a whole byte. Combine first
 * (recoil_combine_splits) to send fewer splits.
 *
 * recoil_serialized_size: *bytes = the container's size, *metadata_bytes (may
 *   be NULL) = the packed metadata section's size. Errors: EINVAL (null, or a
 *   group difference wider than 16 bits / an offset wider than 32 bits).
 * recoil_serialize: writes the container into buf (cap bytes; ENOMEM if too
 *   small) and its size into *written. Errors: EINVAL (also for an adaptive
 *   stream, whose model and table numbers travel with the codec), ENOMEM.
 * recoil_deserialize: parses size bytes at buf into a new stream (freed with
 *   recoil_free), validated as recoil_stream_import does. Errors: EINVAL
 *   (null), ECORRUPT (bad magic, truncated or inconsistent data), ENOMEM.
 */
int recoil_serialized_size(const recoil_stream* s, uint64_t* bytes, uint64_t* metadata_bytes);
int recoil_serialize(const recoil_stream* s, void* buf, uint64_t cap, uint64_t* written);
int recoil_deserialize(const void* buf, uint64_t size, recoil_stream** out);

void recoil_free(recoil_stream* s);
const char* recoil_last_error(void);

/* ------------------------------------------------------------------ device */

/* Batch options. Zero fields take defaults (or the autotuned values). */
typedef struct {
  uint32_t warps_per_cta;    /* decoder warps per CTA (1, 2, 4, 8, 16, 32; adaptive streams 4, 8, 16, 32);
                                0 = about one CTA round of splits per SM: the power of two
                                below splits / SMs, clamped to [4, 16]; adaptive streams with
                                64 or more splits per SM take 32 */
  uint32_t ctas_per_sm;      /* persistent CTAs per SM; default: occupancy maximum */
  uint32_t split_symbols;    /* combine each stream to ceil(N / split_symbols) splits; 0 = keep all */
  uint32_t flags;            /* RECOIL_BATCH_* */
} recoil_batch_opts;

#define RECOIL_BATCH_PER_STREAM 1u   /* one launch per stream (paper-style baseline) instead of one persistent launch */
#define RECOIL_BATCH_NO_SORT 2u      /* keep stream-major item order instead of longest-first */
#define RECOIL_BATCH_GRAPH 4u        /* capture the launch sequence in a CUDA graph on the first
                                        recoil_plan_decode and replay it afterwards (needs a
                                        non-default cuda_stream; ignored with PER_STREAM) */
#define RECOIL_BATCH_NO_PAIRS 8u     /* adaptive models over up to 256 symbols: stage the one-byte
                                        guide layout even where the paired one (one read for the
                                        bracket, one for F and f) fits as well */
#define RECOIL_BATCH_TWO_LANES 16u   /* two coder lanes a thread: each warp decodes two splits at
                                        once, thread j carrying coder j of both (two independent
                                        chains of dependent reads per thread, a word ring per
                                        split); warps_per_cta 4, 8 or 16 for static models, 8, 16
                                        or 24 for adaptive ones; split counts round to whole
                                        CTAs of 2 * warps_per_cta splits */

typedef struct recoil_plan recoil_plan;   /* opaque: device image layout + work queue of a batch */

/*
 * Plan the decode of `count` streams: combine per opts->split_symbols, lay out
 * words, tables and entries for the device, and build the CTA work queue
 * (items of up to warps_per_cta entries of one stream). Host only.
 * The streams must outlive the plan. Errors: EINVAL, ENOMEM.
 */
int recoil_plan_create(const recoil_stream* const* streams, uint32_t count,
                       const recoil_batch_opts* opts, recoil_plan** out);

/* Device bytes the plan needs (workspace), a multiple of 256. */
int recoil_plan_workspace_size(const recoil_plan* plan, size_t* bytes);

/*
 * Copy the plan's device image into d_workspace (>= workspace size bytes,
 * 256-byte aligned, caller-owned) on cuda_stream. Returns once the copies are
 * queued; host sources stay valid while the streams and plan live.
 * Errors: EINVAL (null or too small), ECUDA.
 */
int recoil_plan_upload(recoil_plan* plan, void* d_workspace, size_t ws_bytes, void* cuda_stream);

/*
 * Decode every stream of an uploaded plan: d_outs[i] is a caller-owned device
 * buffer of n_syms * sym_bytes bytes for stream i. One persistent launch (or
 * one launch per stream with RECOIL_BATCH_PER_STREAM), asynchronous on
 * cuda_stream. Kernel-detected inconsistencies are recorded in the workspace
 * and read with recoil_plan_errors. Errors: EINVAL (not uploaded), ECUDA.
 */
int recoil_plan_decode(recoil_plan* plan, void* const* d_outs, void* cuda_stream);

/* Synchronise cuda_stream and read the error flags of the last decode:
 * *flags = 0 when clean. Returns ECORRUPT if any flag is set. */
int recoil_plan_errors(recoil_plan* plan, void* cuda_stream, uint32_t* flags);

/* Number of kernel launches the last recoil_plan_decode issued. */
uint32_t recoil_plan_launches(const recoil_plan* plan);

/* Warps per CTA the plan decodes with (the automatic choice when opts gave 0). */
uint32_t recoil_plan_warps_per_cta(const recoil_plan* plan);

/* Decoder kernels a plan launches, one bit each (host only, no device call). */
#define RECOIL_KERNEL_PACKED8 1u          /* 8-bit symbols, n <= 12: one packed u32 per slot */
#define RECOIL_KERNEL_GENERIC8 2u         /* 8-bit symbols otherwise: slot -> symbol, symbol -> (f, F) */
#define RECOIL_KERNEL_GENERIC16 4u        /* 16-bit symbols, static model otherwise */
#define RECOIL_KERNEL_ADAPTIVE8 8u        /* adaptive, 8-bit symbols, one-byte guide entries */
#define RECOIL_KERNEL_ADAPTIVE16 16u      /* adaptive, 16-bit symbols, alphabet <= 256, one-byte guide entries */
#define RECOIL_KERNEL_ADAPTIVE16_WIDE 32u /* adaptive, alphabet <= 4096, two-byte guide entries */
#define RECOIL_KERNEL_ADAPTIVE8_PAIR 64u  /* adaptive, 8-bit symbols, paired layout */
#define RECOIL_KERNEL_ADAPTIVE16_PAIR 128u /* adaptive, 16-bit symbols, alphabet <= 256, paired layout */
#define RECOIL_KERNEL_PACKED16 256u       /* 16-bit symbols, n <= 15, every f <= 1023: one packed u32 per slot */
uint32_t recoil_plan_kernels(const recoil_plan* plan);

void recoil_plan_free(recoil_plan* plan);

/*
 * Assign streams to `world` ranks (one GPU each) for decoding a batch on
 * several GPUs: longest first (by symbol bytes) to the least-loaded rank,
 * ties to the lower rank. Streams decode independently, so the shards need
 * no exchange while decoding. rank_of[i] receives stream i's rank.
 * Host only. Errors: EINVAL.
 */
int recoil_shard(const recoil_stream* const* streams, uint32_t count, uint32_t world, uint32_t* rank_of);

/*
 * One stream over `world` ranks (one GPU each): the stream's kept entries are
 * cut into `world` contiguous runs of about equal owned symbols, and rank
 * `rank` gets a plan that decodes only its run. Each run owns a contiguous
 * symbol range [*sym_lo, *sym_hi) (Sec. 4.1.3 ownership), the ranges of all
 * ranks tile [0, N), and the runs share nothing, so the ranks decode with no
 * exchange; the result is the concatenation of the ranges. Combine first
 * (recoil_combine_splits) to choose the split count. opts as for
 * recoil_plan_create (its split_symbols must be 0). The plan's decode takes
 * one output pointer to a buffer of (*sym_hi - *sym_lo) * sym_bytes bytes
 * that receives symbols *sym_lo ..; the workspace holds the whole stream's
 * words. A rank whose run is empty gets sym_lo == sym_hi and a plan that
 * launches nothing. Errors: EINVAL (null, world < 1, rank >= world,
 * split_symbols set), ENOMEM.
 */
int recoil_plan_create_shard(const recoil_stream* stream, uint32_t world, uint32_t rank,
                             const recoil_batch_opts* opts, recoil_plan** out, uint64_t* sym_lo,
                             uint64_t* sym_hi);

/* Workspace bytes recoil_decode_batch needs for these streams and options. */
int recoil_workspace_size(const recoil_stream* const* streams, uint32_t count,
                          const recoil_batch_opts* opts, size_t* bytes);

/*
 * Decode one stream into d_out (caller-owned device buffer of
 * n_syms * sym_bytes bytes): plan, upload into d_workspace, and launch, all
 * on cuda_stream. Same as recoil_decode_batch with count = 1.
 */
int recoil_decode(const recoil_stream* stream, void* d_out, void* d_workspace, size_t ws_bytes,
                  void* cuda_stream);

/*
 * Decode many streams of uneven sizes, each with its own table, in one
 * persistent launch fed by a device work queue (plan + upload + decode).
 * Errors: as the plan functions.
 */
int recoil_decode_batch(const recoil_stream* const* streams, uint32_t count, void* const* d_outs,
                        void* d_workspace, size_t ws_bytes, void* cuda_stream,
                        const recoil_batch_opts* opts);

/* ------------------------------------------------- host-to-host pipeline */

typedef struct recoil_pipeline recoil_pipeline;   /* opaque: grouped plans + copy/compute streams */

/*
 * Prepare host-to-host decoding of `count` streams with copy/compute overlap:
 * the streams are cut into `groups` (0 = 8) groups of about equal output
 * bytes -- a stream larger than that share is cut into runs of its splits
 * (recoil_plan_create_shard), so even one stream overlaps copies and
 * decoding -- each with its own plan (opts as for recoil_plan_create), a page-
 * locked copy of its descriptors and a page-locked image of its words, table
 * numbers and tables as they lie in the workspace (so a group is copied in
 * with two copies; the pipeline holds about the streams' compressed size in
 * page-locked host memory). The streams must outlive the pipeline.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
int recoil_pipeline_create(const recoil_stream* const* streams, uint32_t count, const recoil_batch_opts* opts,
                           uint32_t groups, recoil_pipeline** out);

/* Device bytes a run needs: the workspace and the staging buffer for the symbols. */
int recoil_pipeline_sizes(const recoil_pipeline* p, size_t* ws_bytes, size_t* staging_bytes);

/*
 * Decode every stream into host memory: h_outs[i] receives n_syms * sym_bytes
 * bytes (page-locked for full link speed; buffers of consecutive streams that
 * follow each other in memory are copied out together). Per group, on three internal CUDA
 * streams: copy the group in, decode it, copy its symbols out, so copies in
 * both directions overlap the decoding of other groups. The run starts after
 * work already queued on cuda_stream and cuda_stream waits for its end, so
 * synchronising cuda_stream (or an event recorded on it) ends the run.
 * d_ws and d_staging: caller device buffers of at least the sizes above,
 * 256-byte aligned. Errors: EINVAL, ENOMEM, ECUDA.
 */
int recoil_pipeline_run(recoil_pipeline* p, void* const* h_outs, void* d_ws, size_t ws_bytes, void* d_staging,
                        size_t staging_bytes, void* cuda_stream);

/* After a run has finished: error flags of its decodes (ECORRUPT if any). */
int recoil_pipeline_errors(recoil_pipeline* p, uint32_t* flags);

void recoil_pipeline_free(recoil_pipeline* p);

/* -------------------------------------------------------------- serving */

typedef struct {
  size_t budget_bytes;       /* device memory admitted requests' outputs may use at once (e.g. 20 GiB) */
  uint32_t max_inflight;     /* launches on the device at once, each on its own CUDA stream (default 8) */
  uint32_t max_batch;        /* requests admitted into one launch (default 64; up to 8x that when
                                more than max_batch requests have arrived and wait) */
  uint32_t warps_per_cta;    /* default 8 (4 with RECOIL_SERVE_PER_REQUEST) */
  uint32_t flags;            /* RECOIL_SERVE_* */
  size_t meta_bytes;         /* descriptor area per launch (default 16 MiB) */
  double timeout_s;          /* wall-clock limit of the run (default 60 s) */
  uint32_t max_split_symbols; /* longest split a request is combined to (default 131072): a
                                 split is one warp's sequential work, so this bounds latency */
  uint32_t reserved;
} recoil_serve_opts;

#define RECOIL_SERVE_PER_REQUEST 1u  /* baseline: one launch per request with every encoded split, one at a time */

typedef struct {
  double arrival_s;          /* request arrival, seconds from the start of the run */
  double admit_s;            /* when the loop admitted it */
  double done_s;             /* device completion of the launch that carried it */
  uint32_t splits;           /* split count it was decoded with */
  uint32_t launch;           /* index of that launch */
} recoil_request_result;

typedef struct {
  uint64_t requests;
  uint64_t launches;
  uint64_t symbol_bytes;     /* decoded bytes over all requests */
  double makespan_s;         /* first arrival to last completion */
  double decoded_gbs;        /* symbol_bytes / makespan */
  double p50_ms, p99_ms, mean_ms;   /* latency = done - arrival */
  uint32_t max_inflight;     /* most launches seen on the device at once */
} recoil_serve_stats;

/* Arena bytes recoil_serve needs: resident pool words, tables and split
 * descriptors (every entry of every pool stream, 288 bytes each), one
 * descriptor area per launch slot, and the output budget. */
int recoil_serve_arena_size(const recoil_stream* const* pool, uint32_t pool_count, const recoil_serve_opts* opts,
                            size_t* bytes);

/*
 * Serve decode requests with continuous batching on the current GPU (the
 * content-delivery setting of Sec. 3.3: each request is combined to the
 * parallelism the decoder has when it is admitted). The pool's words,
 * tables and split descriptors are uploaded once into d_arena (resident);
 * an admission sends 16 bytes per kept split. Request r asks for pool
 * stream req_stream[r] at req_arrival_s[r] (seconds from the start, non-
 * decreasing) and is replayed in real time. Arrived requests are admitted in
 * order while the budget and a launch slot allow, combined to their share of
 * the free warp slots (but to at least n_syms / max_split_symbols splits, so
 * that a large request admitted into a busy device is not left with a few
 * long splits), and launched together as one persistent decode on the
 * slot's CUDA stream; launches overlap on the device. Outputs go to
 * d_req_outs[r] (caller device buffers of n_syms * sym_bytes) or, with
 * d_req_outs NULL, to arena memory that is reused once a request completes.
 * results[r] receives the timeline of request r, *stats the summary (may be
 * NULL). Returns when every request has completed. Errors: EINVAL, ENOMEM
 * (arena or descriptor area too small), ECORRUPT, ETIMEOUT (timeout_s passed;
 * the launches already made are finished first), ECUDA.
 */
int recoil_serve(const recoil_stream* const* pool, uint32_t pool_count, const uint32_t* req_stream,
                 const double* req_arrival_s, uint32_t n_req, void* d_arena, size_t arena_bytes,
                 void* const* d_req_outs, const recoil_serve_opts* opts, recoil_request_result* results,
                 recoil_serve_stats* stats);

/* ----------------------------------------------------------- autotuning */

typedef struct {
  uint32_t steps;            /* timed decodes per candidate (default 3) */
  uint32_t flags;            /* RECOIL_TUNE_* */
  const char* cache_path;    /* text file of tuned results, or NULL for none */
} recoil_tune_opts;

#define RECOIL_TUNE_REFRESH 1u     /* ignore a cached result and tune again */
#define RECOIL_TUNE_KEEP_SPLITS 2u /* keep the streams' split counts; tune warps_per_cta only */

/* Workspace bytes recoil_autotune needs for these streams (the largest candidate). */
int recoil_autotune_workspace_size(const recoil_stream* const* streams, uint32_t count, size_t* bytes);

/*
 * Choose batch options for these streams by measurement (the batching pattern
 * of the paper's decoder-adaptive parallelism, Sec. 3.3: the decoder picks the
 * split count that suits it). Candidates: coder lanes a thread (one, or two
 * with RECOIL_BATCH_TWO_LANES) times the warps_per_cta built for that and for
 * every kind in the batch (one lane: 4, 8, 16, and 32 when a stream is
 * adaptive or has 16-bit symbols; two lanes: 4, 8, 16 static, 8, 16, 24
 * adaptive) times
 * split_symbols in {32 Ki, 64 Ki, 128 Ki, 256 Ki} (with
 * RECOIL_TUNE_KEEP_SPLITS: split_symbols 0, the streams as given, for a
 * decoder whose split count is already chosen), and, when an adaptive model
 * has at most 256 symbols, both table layouts (paired, or the one-byte guide
 * with RECOIL_BATCH_NO_PAIRS). Each candidate decodes the streams into d_outs
 * (caller-owned, as for recoil_plan_decode) once untimed and `steps` times
 * timed with CUDA events on cuda_stream; the lowest median wins and is
 * written to *best (ctas_per_sm = 0; flags: the winner's
 * RECOIL_BATCH_TWO_LANES and RECOIL_BATCH_NO_PAIRS bits) with its time in
 * *best_ms (may be NULL). With a cache_path, a result cached for the same GPU
 * and batch shape is returned without decoding, and new results are appended
 * (one line: key, warps, split symbols, lanes, layout 0 or 1, ms).
 * d_workspace: >= recoil_autotune_workspace_size bytes, 256-byte aligned.
 * Synchronises cuda_stream. Errors: EINVAL, ENOMEM (workspace too small),
 * ECORRUPT, ECUDA.
 */
int recoil_autotune(const recoil_stream* const* streams, uint32_t count, void* const* d_outs, void* d_workspace,
                    size_t ws_bytes, void* cuda_stream, const recoil_tune_opts* opts, recoil_batch_opts* best,
                    float* best_ms);

/* --------------------------------------------------------- no allocation */

/* Device bytes the library keeps for recoil_decode_noalloc (per GPU, for the
 * life of the process). */
#define RECOIL_NOALLOC_SCRATCH_BYTES (4u << 20)

/*
 * Decode one stream without any device allocation. The paper has no
 * counterpart: this exists for callers that cannot call cudaMalloc (or any
 * allocator built on it) where they decode -- code inside a host framework
 * that owns all device memory and only lends fixed buffers, or a path where an
 * allocation might block or fail at the wrong moment. Such a caller passes
 * device buffers it already holds:
 *   d_words      the stream's 16-bit words (recoil_stream_export order),
 *                16-byte aligned, in a buffer of words_bytes >=
 *                ceil(n_words / 256) * 512 bytes (the tail is never used as data)
 *   d_out        n_syms * sym_bytes bytes for the symbols
 * The split descriptors, decoder tables, work-queue counters and error flags
 * go to one static device array of RECOIL_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until exit; each call looks up its device address
 * on the current device. Every call shares the array and finds the previous
 * call's contents there; a call clears the counters and flags it needs, but
 * calls whose GPU work overlaps (several host threads or CUDA streams) race on
 * it and must not be made. Allocates nothing on the device (host memory only
 * for building the descriptors). Synchronous: it copies the descriptors from
 * host memory, waits on cuda_stream and returns after the decode has finished
 * (also on an error return, nothing it queued is still running). Errors: EINVAL (null, small or misaligned d_words, an adaptive
 * stream, or a stream whose descriptors and tables exceed the array: combine
 * it to fewer splits),
 * ECORRUPT (the decoder found an inconsistent stream), ECUDA.
 */
int recoil_decode_noalloc(const recoil_stream* stream, const void* d_words, size_t words_bytes, void* d_out,
                          void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RECOIL_H */
