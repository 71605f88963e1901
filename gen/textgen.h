/*
 * Seeded, counter-based input generators shared by the test/bench harness.
 *
 * This header holds NO string-matching arithmetic: it only turns (key, index)
 * into pseudo-random bytes.  The same inline functions are compiled by gcc for
 * the host (gen_host.c) and by nvcc for the device (gen_cuda.cu), so a text made
 * on the GPU is byte-identical to the one made on the CPU for the same seed.
 *
 * Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) used in counter mode: draw(key, i) =
 * mix64(key + (i + 1) * GOLDEN), where mix64 is the published finaliser.
 */
#ifndef EPSM_TEXTGEN_H
#define EPSM_TEXTGEN_H

#include <stdint.h>

#if defined(__CUDACC__)
#define GEN_HD __host__ __device__ __forceinline__
#else
#define GEN_HD static inline
#endif

#define GEN_GOLDEN 0x9E3779B97F4A7C15ULL

GEN_HD uint64_t gen_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* 64 random bits for counter i under key. */
GEN_HD uint64_t gen_draw(uint64_t key, uint64_t i) {
    return gen_mix64(key + (i + 1ULL) * GEN_GOLDEN);
}

/* Key for a (seed, stream) pair; streams separate independent uses of a seed. */
GEN_HD uint64_t gen_key(uint64_t seed, uint64_t stream) {
    return gen_mix64(gen_mix64(seed + GEN_GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL + 1ULL));
}

/* 16 random bits for byte index i: four bytes share one 64-bit draw. */
GEN_HD uint32_t gen_u16(uint64_t key, uint64_t i) {
    return (uint32_t)((gen_draw(key, i >> 2) >> (16u * (uint32_t)(i & 3u))) & 0xFFFFu);
}

/* i.i.d. text: byte i = table[u16(key, i)] (table has 65536 entries). */
GEN_HD uint8_t gen_iid_byte(uint64_t key, uint64_t i, const uint8_t *table) {
    return table[gen_u16(key, i)];
}

/* Order-2 Markov text, generated in independent segments of GEN_MARKOV_SEG
 * bytes so that any range can be produced in parallel.  A segment starts from
 * two symbols drawn from the 96-symbol start table; every later byte is drawn
 * from the 1024-entry row of its two-symbol context. */
#define GEN_MARKOV_SEG 65536ULL
#define GEN_MARKOV_NSYM 96
#define GEN_MARKOV_ROW 1024

/* Advance a Markov segment from its start to (exclusive) local index `upto`,
 * writing bytes [from, upto) of the segment to dst[0 ..).  sym_index maps a byte
 * to its 0..95 symbol index; rows is [96*96][1024] symbol bytes. */
GEN_HD void gen_markov_segment(uint64_t key, uint64_t seg, uint64_t from, uint64_t upto,
                               const uint8_t *start_table, const uint8_t *rows,
                               const uint8_t *sym_index, uint8_t *dst) {
    uint64_t base = seg * GEN_MARKOV_SEG;
    uint8_t a = start_table[gen_u16(key, base) & 0xFFFFu];
    uint8_t b = start_table[gen_u16(key, base + 1) & 0xFFFFu];
    for (uint64_t j = 0; j < upto; ++j) {
        uint8_t c;
        if (j == 0) c = a;
        else if (j == 1) c = b;
        else {
            uint32_t ctx = (uint32_t)sym_index[a] * GEN_MARKOV_NSYM + sym_index[b];
            c = rows[(uint64_t)ctx * GEN_MARKOV_ROW + (gen_u16(key, base + j) & (GEN_MARKOV_ROW - 1))];
            a = b;
            b = c;
        }
        if (j >= from) dst[j - from] = c;
    }
}

/* Adversarial runs: the text is cut into blocks of `block` bytes; in block B one
 * run of `run_byte` starts at a random offset with a random length in
 * [1, maxlen], clipped at the block end.  Returns whether byte i is in a run. */
GEN_HD int gen_in_run(uint64_t key, uint64_t i, uint64_t block, uint32_t maxlen) {
    uint64_t B = i / block;
    uint64_t d = gen_draw(key, B);
    uint64_t start = (d & 0xFFFFFFFFULL) % block;
    uint64_t len = 1 + ((d >> 32) % maxlen);
    uint64_t off = i - B * block;
    return off >= start && off < start + len;
}

#endif /* EPSM_TEXTGEN_H */
