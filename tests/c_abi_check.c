/*
 * Plain C11 user of include/recoil.h (compiled and run by test_c_abi.py): the
 * header must compile as C and the library must serve the host-side entry
 * points to a C caller. Encodes a byte sequence with splits under both T
 * rules of Def. 4.1 / Eq. 7, combines, exports, serialises and
 * deserialises, imports the exported parts, and plans a decode (host only),
 * checking sizes and error codes along the way. Prints "ok" on success.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "recoil.h"

#define CHECK(cond)                                                         \
  do {                                                                      \
    if (!(cond)) {                                                          \
      fprintf(stderr, "failed: %s (line %d): %s\n", #cond, __LINE__,        \
              recoil_last_error());                                         \
      return 1;                                                             \
    }                                                                       \
  } while (0)

int main(void) {
  enum { N = 100003 };
  uint8_t* syms = (uint8_t*)malloc(N);
  uint32_t r = 12345u;
  for (int i = 0; i < N; i++) {           /* a skewed byte source */
    r = r * 1103515245u + 12345u;
    syms[i] = (uint8_t)((r >> 16) % 7 == 0 ? (r >> 8) & 0xff : (r >> 20) & 0x0f);
  }
  recoil_params p;
  memset(&p, 0, sizeof p);
  p.n_bits = 12;
  p.sym_bytes = 1;

  recoil_stream* s = NULL;
  CHECK(recoil_encode_with_splits(syms, N, &p, 64, &s) == RECOIL_OK);
  recoil_info info;
  CHECK(recoil_stream_info(s, &info) == RECOIL_OK);
  CHECK(info.n_syms == N && info.n_entries == 64 && info.n_bits == 12 && info.sym_bytes == 1);

  /* the printed T = ceil(N / M) places other split words on this source */
  recoil_params pe = p;
  pe.split_rule = RECOIL_SPLIT_EQ7;
  recoil_stream* se = NULL;
  CHECK(recoil_encode_with_splits(syms, N, &pe, 64, &se) == RECOIL_OK);
  recoil_info ie;
  CHECK(recoil_stream_info(se, &ie) == RECOIL_OK);
  CHECK(ie.n_words == info.n_words);       /* same bitstream, other metadata */
  pe.split_rule = 7;
  recoil_stream* bad = NULL;
  CHECK(recoil_encode_with_splits(syms, N, &pe, 64, &bad) == RECOIL_EINVAL && bad == NULL);

  recoil_stream* c = NULL;
  CHECK(recoil_combine_splits(s, 16, &c) == RECOIL_OK);
  recoil_info ic;
  CHECK(recoil_stream_info(c, &ic) == RECOIL_OK && ic.n_entries == 16 && ic.n_words == info.n_words);

  /* export and import the parts: the same stream */
  const uint32_t R = info.n_entries - 1;
  uint32_t* freq = (uint32_t*)calloc(info.alphabet, 4);
  uint16_t* words = (uint16_t*)calloc(info.n_words ? info.n_words : 1, 2);
  uint32_t fin[RECOIL_W];
  uint64_t* ew = (uint64_t*)calloc(R ? R : 1, 8);
  uint64_t* ei = (uint64_t*)calloc((size_t)(R ? R : 1) * RECOIL_W, 8);
  uint16_t* es = (uint16_t*)calloc((size_t)(R ? R : 1) * RECOIL_W, 2);
  CHECK(recoil_stream_export(s, freq, words, fin, ew, ei, es) == RECOIL_OK);
  recoil_stream* im = NULL;
  CHECK(recoil_stream_import(&p, N, info.alphabet, freq, words, info.n_words, fin, R, ew, ei, es, &im) ==
        RECOIL_OK);
  recoil_info ii;
  CHECK(recoil_stream_info(im, &ii) == RECOIL_OK && ii.n_entries == info.n_entries);
  ew[1] = ew[0]; /* split words must strictly increase: validation refuses the parts */
  recoil_stream* im2 = NULL;
  CHECK(recoil_stream_import(&p, N, info.alphabet, freq, words, info.n_words, fin, R, ew, ei, es, &im2) < 0 &&
        im2 == NULL);

  /* packed metadata (Sec. 4.3) round trip */
  uint64_t bytes = 0, meta = 0, written = 0;
  CHECK(recoil_serialized_size(c, &bytes, &meta) == RECOIL_OK && bytes > meta && meta > 0);
  uint8_t* buf = (uint8_t*)malloc(bytes);
  CHECK(recoil_serialize(c, buf, bytes, &written) == RECOIL_OK && written == bytes);
  recoil_stream* d = NULL;
  CHECK(recoil_deserialize(buf, written, &d) == RECOIL_OK);
  recoil_info id;
  CHECK(recoil_stream_info(d, &id) == RECOIL_OK && id.n_entries == 16 && id.n_syms == N);

  /* a plan is host work: its workspace size needs no device */
  recoil_batch_opts o;
  memset(&o, 0, sizeof o);
  o.warps_per_cta = 8;
  o.flags = RECOIL_BATCH_GRAPH;
  const recoil_stream* one[2] = {s, d};
  recoil_plan* plan = NULL;
  CHECK(recoil_plan_create(one, 2, &o, &plan) == RECOIL_OK);
  size_t ws = 0;
  CHECK(recoil_plan_workspace_size(plan, &ws) == RECOIL_OK && ws > 2 * info.n_words);
  CHECK(recoil_plan_kernels(plan) == RECOIL_KERNEL_PACKED8 && recoil_plan_warps_per_cta(plan) == 8);
  recoil_plan_free(plan);
  o.flags = RECOIL_BATCH_TWO_LANES;
  o.warps_per_cta = 32;                     /* no two-lane kernel has 32 warps */
  CHECK(recoil_plan_create(one, 2, &o, &plan) == RECOIL_EINVAL && plan == NULL);

  CHECK(recoil_combine_splits(NULL, 4, &bad) == RECOIL_EINVAL);
  recoil_free(d);
  recoil_free(im);
  recoil_free(c);
  recoil_free(se);
  recoil_free(s);
  free(buf);
  free(es);
  free(ei);
  free(ew);
  free(words);
  free(freq);
  free(syms);
  printf("ok\n");
  return 0;
}
