/*
 * CPU oracle for exact string matching (test infrastructure only).
 *
 * This file is the checker, not the product: only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  The GPU library never
 * links or calls it, and it shares no code, header or table with the GPU path.
 *
 * What it computes (Section 1 and Section 2 of the paper): given a text t[0..n-1]
 * and a pattern p[0..m-1] over bytes, the exact string matching problem asks for
 * ALL start positions s, 0 <= s <= n-m, with t[s+i] == p[i] for every i < m.
 * Overlapping occurrences are all reported; positions are 0-based and ascending.
 * Characters are compared as unsigned bytes (sigma = 256, Section 3.1).
 *
 * The paper's EPSM procedures (EPSMa/EPSMb/EPSMc, Section 3) are exact: every
 * filter hit is followed by a naive check.  The result therefore has a plain
 * definition, and this oracle is that definition written out as a brute-force
 * O(nm) scan with an explicit byte loop.  A second, independent counter (the
 * Knuth-Morris-Pratt automaton, cited in Section 1 as the classical O(n) method)
 * is provided so the scan can be pinned against a different algorithm.
 *
 * Parity pins: see the not-gpu oracle tests (closed forms, exhaustive tiny
 * inputs, planted occurrences, library string routines, KMP).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_API __attribute__((visibility("default")))

/* Brute-force scan of start positions [s_begin, s_end) (Section 1 definition).
 * Writes at most `cap` positions to `out` (may be NULL when cap == 0) and
 * returns the number of occurrences in the range. */
static uint64_t scan_range(const uint8_t *t, uint64_t n, const uint8_t *p,
                           uint32_t m, uint64_t s_begin, uint64_t s_end,
                           uint64_t *out, uint64_t cap) {
    uint64_t count = 0;
    if (m == 0 || m > n) return 0;
    if (s_end > n - m + 1) s_end = n - m + 1;
    for (uint64_t s = s_begin; s < s_end; ++s) {
        uint32_t i = 0;
        while (i < m && t[s + i] == p[i]) ++i;
        if (i == m) {
            if (count < cap) out[count] = s;
            ++count;
        }
    }
    return count;
}

/* All occurrences of p in t, ascending.  Returns the true count; writes the
 * first min(count, cap) positions. m == 0 returns 0 (the paper defines m > 0). */
ORACLE_API uint64_t oracle_search(const uint8_t *t, uint64_t n, const uint8_t *p,
                                  uint32_t m, uint64_t *out, uint64_t cap) {
    if (m == 0 || m > n) return 0;
    return scan_range(t, n, p, m, 0, n - m + 1, out, cap);
}

ORACLE_API uint64_t oracle_count(const uint8_t *t, uint64_t n, const uint8_t *p,
                                 uint32_t m) {
    return oracle_search(t, n, p, m, NULL, 0);
}

/* ---- multithreaded form: the start range is split into contiguous parts; each
 * part is counted, the counts are prefix-summed, and each part then writes its
 * positions at its offset.  Same definition, only the range is partitioned. */
typedef struct {
    const uint8_t *t; uint64_t n; const uint8_t *p; uint32_t m;
    uint64_t s0, s1; uint64_t *out; uint64_t cap; uint64_t offset; uint64_t count;
    int fill;
} part_t;

static void *part_main(void *arg) {
    part_t *w = (part_t *)arg;
    if (!w->fill) {
        w->count = scan_range(w->t, w->n, w->p, w->m, w->s0, w->s1, NULL, 0);
    } else if (w->offset < w->cap) {
        scan_range(w->t, w->n, w->p, w->m, w->s0, w->s1, w->out + w->offset,
                   w->cap - w->offset);
    }
    return NULL;
}

ORACLE_API uint64_t oracle_search_mt(const uint8_t *t, uint64_t n, const uint8_t *p,
                                     uint32_t m, uint64_t *out, uint64_t cap,
                                     int nthreads) {
    if (m == 0 || m > n) return 0;
    uint64_t starts = n - m + 1;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > starts) nthreads = (int)starts;
    if (nthreads == 1) return oracle_search(t, n, p, m, out, cap);
    part_t *parts = (part_t *)calloc((size_t)nthreads, sizeof(part_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!parts || !th) { free(parts); free(th); return oracle_search(t, n, p, m, out, cap); }
    for (int k = 0; k < nthreads; ++k) {
        parts[k].t = t; parts[k].n = n; parts[k].p = p; parts[k].m = m;
        parts[k].s0 = starts * (uint64_t)k / (uint64_t)nthreads;
        parts[k].s1 = starts * (uint64_t)(k + 1) / (uint64_t)nthreads;
        parts[k].out = out; parts[k].cap = cap; parts[k].fill = 0;
    }
    for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, part_main, &parts[k]);
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    uint64_t total = 0;
    for (int k = 0; k < nthreads; ++k) { parts[k].offset = total; total += parts[k].count; }
    if (cap > 0 && out != NULL) {
        for (int k = 0; k < nthreads; ++k) { parts[k].fill = 1; pthread_create(&th[k], NULL, part_main, &parts[k]); }
        for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    }
    free(parts); free(th);
    return total;
}

/* ---- independent counter: Knuth-Morris-Pratt (Section 1 cites it as the
 * classical linear-time method).  Written from the textbook definition of the
 * failure function: fail[i] = length of the longest proper border of p[0..i].
 * Counts overlapping occurrences by falling back to fail[m-1] after a match. */
ORACLE_API uint64_t oracle_kmp_count(const uint8_t *t, uint64_t n, const uint8_t *p,
                                     uint32_t m) {
    if (m == 0 || m > n) return 0;
    uint32_t *fail = (uint32_t *)malloc(sizeof(uint32_t) * m);
    if (!fail) return UINT64_MAX;
    fail[0] = 0;
    uint32_t k = 0;
    for (uint32_t i = 1; i < m; ++i) {
        while (k > 0 && p[i] != p[k]) k = fail[k - 1];
        if (p[i] == p[k]) ++k;
        fail[i] = k;
    }
    uint64_t count = 0;
    uint32_t q = 0; /* length of the current matched prefix */
    for (uint64_t j = 0; j < n; ++j) {
        while (q > 0 && t[j] != p[q]) q = fail[q - 1];
        if (t[j] == p[q]) ++q;
        if (q == m) { ++count; q = fail[m - 1]; }
    }
    free(fail);
    return count;
}
