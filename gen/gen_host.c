/* Host side of the seeded input generators (see textgen.h).  Holds no
 * string-matching arithmetic; produces the same bytes as gen_cuda.cu. */
#include <stdint.h>
#include <string.h>
#include "textgen.h"

#define GEN_API __attribute__((visibility("default")))

/* Bytes [start, start+len) of an i.i.d. text. */
GEN_API void gen_fill_iid(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                          const uint8_t *table) {
    for (uint64_t i = 0; i < len; ++i) dst[i] = gen_iid_byte(key, start + i, table);
}

/* Bytes [start, start+len) of a segmented order-2 Markov text. */
GEN_API void gen_fill_markov(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                             const uint8_t *start_table, const uint8_t *rows,
                             const uint8_t *sym_index) {
    uint64_t end = start + len;
    uint64_t pos = start;
    while (pos < end) {
        uint64_t seg = pos / GEN_MARKOV_SEG;
        uint64_t seg_base = seg * GEN_MARKOV_SEG;
        uint64_t from = pos - seg_base;
        uint64_t upto = end - seg_base;
        if (upto > GEN_MARKOV_SEG) upto = GEN_MARKOV_SEG;
        gen_markov_segment(key, seg, from, upto, start_table, rows, sym_index,
                           dst + (pos - start));
        pos = seg_base + upto;
    }
}

/* Overwrite the run bytes inside [start, start+len) with run_byte. */
GEN_API void gen_apply_runs(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                            uint64_t block, uint32_t maxlen, uint8_t run_byte) {
    for (uint64_t i = 0; i < len; ++i)
        if (gen_in_run(key, start + i, block, maxlen)) dst[i] = run_byte;
}
