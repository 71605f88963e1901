// Per-chunk filters and verify of the three length regimes (Section 3).
//
// A chunk is 16 text bytes held as four little-endian 32-bit words; a lane
// also sees the next chunk (its neighbour lane's, by a shuffle).  For each
// chunk a 16-bit mask marks hits: bit i <-> internal start pos0 + OFF + i,
// with pos0 = 16*chunk.  OFF = 0 for the window variants; the 8-byte block
// variant reports candidate s = 8b - j from block b, j in [0, 8), so a
// chunk's two blocks cover starts [pos0 - 7, pos0 + 8] and OFF = -7.  The
// 4-byte block variant looks at the chunk's words and the next chunk's first
// one (k = 0..4) and reports s = 4k - j for s in [pos0, pos0 + 15]: OFF = 0.
#pragma once

#include "epsm_scan.cuh"

namespace epsm {

// Pattern preprocessing for the block variants (Section 3.4, table L): the
// fingerprints of the pattern blocks p[j..j+7], j < nb (8 for the plain block
// variant; 16 for the strided one, whose inspected blocks lie at j = 0..15 of
// an occurrence), marked in the bit table, and the blocks themselves in pblk
// (2 * nb words).  Must be called by all threads of the block; ends with a
// barrier.
__device__ __forceinline__ void build_block_table(const Pattern &pat, uint32_t *table,
                                                  uint32_t *pblk, int nb) {
    for (int i = threadIdx.x; i < kTableWords; i += blockDim.x) table[i] = 0u;
    __syncthreads();
    if ((int)threadIdx.x < nb) {
        const int j = threadIdx.x;
        const int q = j >> 2;
        const uint32_t sh = 8u * (uint32_t)(j & 3);
        const uint32_t lo = __funnelshift_r(pat.w[q], pat.w[q + 1], sh);
        const uint32_t hi = __funnelshift_r(pat.w[q + 1], pat.w[q + 2], sh);
        pblk[2 * j] = lo;
        pblk[2 * j + 1] = hi;
        const uint32_t h = block_hash(lo, hi, pat.kbits);
        atomicOr(&table[h >> 5], 1u << (h & 31u));
    }
    __syncthreads();
}

// Broadcast words (p_j)^4 of the first eight pattern bytes (Section 3.2, table B).
struct BcastWords {
    uint32_t b[8];
    uint32_t r2[8];  // the 2-bit code of p_j replicated 16 times (2-bit code variant)
    __device__ __forceinline__ explicit BcastWords(const Pattern &pat) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            b[j] = bcast_byte(pat.w[j >> 2], j & 3);
            r2[j] = ((b[j] >> 1) & 0x03030303u) * 0x55u;
        }
    }
};

// Mismatch word of a 4-byte pattern piece at the 4 starts of word R0 (R1 next):
// byte k is zero iff t[4w+k .. 4w+k+3] equals the piece (b0..b3 broadcast).
template <int NB>
__device__ __forceinline__ uint32_t window_mismatch(uint32_t acc, uint32_t R0, uint32_t R1,
                                                    uint32_t b0, uint32_t b1, uint32_t b2,
                                                    uint32_t b3) {
    acc |= R0 ^ b0;
    if (NB > 1) acc |= __funnelshift_r(R0, R1, 8) ^ b1;
    if (NB > 2) acc |= __funnelshift_r(R0, R1, 16) ^ b2;
    if (NB > 3) acc |= __funnelshift_r(R0, R1, 24) ^ b3;
    return acc;
}

// 16-bit mask of bits [lo, hi] (clipped to 0..15); 0 if empty.
__device__ __forceinline__ uint32_t range_mask(int64_t lo, int64_t hi) {
    if (hi < 0 || lo > 15 || lo > hi) return 0u;
    int a = lo < 0 ? 0 : (int)lo;
    int b = hi > 15 ? 15 : (int)hi;
    return (0xFFFFu >> (15 - b)) & (0xFFFFu << a) & 0xFFFFu;
}

// In-register verify of pattern words [w_from, nw) for the start at byte b of
// word K of the chunk; RR holds the chunk's words and the next chunk's words.
template <int K>
__device__ __forceinline__ bool verify_regs(const uint32_t (&RR)[8], uint32_t b, uint32_t w_from,
                                            const Pattern &pat) {
    uint32_t m = pat.m;
    uint32_t nw = (m + 3u) >> 2;
    bool ok = true;
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        if ((uint32_t)i >= w_from && (uint32_t)i < nw) {
            uint32_t win = __funnelshift_r(RR[K + i], RR[K + i + 1], 8u * b);
            ok &= ((win ^ pat.w[i]) & word_mask(m, (uint32_t)i)) == 0u;
        }
    }
    return ok;
}

template <int K>
__device__ __forceinline__ uint32_t verify_word_hits(uint32_t z, const uint32_t (&RR)[8],
                                                     uint32_t w_from, const Pattern &pat) {
    uint32_t h = 0u;
    while (z) {
        uint32_t b = (uint32_t)(__ffs(z) >> 3) - 1u;
        z &= z - 1u;
        if (verify_regs<K>(RR, b, w_from, pat)) h |= 1u << (4 * K + b);
    }
    return h;
}

// Exact check of all 16 starts of a chunk at once, for chunks with many
// candidates (runs of one byte and the like), given the text as words R[0..]
// aligned to the chunk's first start (R must hold 16 + m - 1 bytes): for every
// pattern byte j the shifted text words are XORed with (p_j)^4 and ORed into
// one mismatch word per 4 starts, whose zero bytes are the hits (the
// packed compare of Section 3.2 extended to every j < m).
template <int NW>
__device__ __forceinline__ uint32_t exact_starts16(const uint32_t (&R)[NW], const Pattern &pat) {
    static_assert(NW >= 5 && NW <= 12, "16 starts and up to 32 pattern bytes");
    uint32_t acc0 = 0u, acc1 = 0u, acc2 = 0u, acc3 = 0u;
    const uint32_t m = pat.m;
#pragma unroll
    for (int j = 0; j < 4 * (NW - 4); ++j) {
        if ((uint32_t)j < m) {
            const uint32_t b = bcast_byte(pat.w[j >> 2], j & 3);
            const int q = j >> 2, sh = 8 * (j & 3);
            acc0 |= (sh ? __funnelshift_r(R[q], R[q + 1], sh) : R[q]) ^ b;
            acc1 |= (sh ? __funnelshift_r(R[q + 1], R[q + 2], sh) : R[q + 1]) ^ b;
            acc2 |= (sh ? __funnelshift_r(R[q + 2], R[q + 3], sh) : R[q + 2]) ^ b;
            acc3 |= (sh ? __funnelshift_r(R[q + 3], R[q + 4], sh) : R[q + 3]) ^ b;
        }
    }
    return nibble_of(zero_bytes(acc0)) | (nibble_of(zero_bytes(acc1)) << 4) |
           (nibble_of(zero_bytes(acc2)) << 8) | (nibble_of(zero_bytes(acc3)) << 12);
}

// exact_starts16 on the bytes of a chunk and the next chunk (m <= 16); out
// of line, so the filter loops that rarely call it keep their registers.
__device__ __noinline__ uint32_t exact_chunk_regs(const Pattern &pat, const uint4 cur, uint32_t n0,
                                                  uint32_t n1, uint32_t n2, uint32_t n3) {
    const uint32_t R[8] = {cur.x, cur.y, cur.z, cur.w, n0, n1, n2, n3};
    return exact_starts16<8>(R, pat);
}

// Exact hits of the 16 starts p0 .. p0+15 for a pattern that is one byte
// repeated m times (period 1), from text words R[] aligned at p0 that hold at
// least 15 + m bytes.  With E the mask of the text bytes equal to that byte
// (Section 3.2's packed compare against the broadcast byte: one compare per
// text word whatever m is), start i is an occurrence iff bits i .. i+m-1 of E
// are all set; doubling shift-ANDs find those runs of m ones in log2 m steps.
// A run of that byte in the text makes every start a candidate of the
// fingerprint and code filters; this decides a chunk's 16 starts at once.
// Bits i (0..15) such that bits i .. i+m-1 of E are all set (1 <= m <= 48).
__device__ __forceinline__ uint32_t runs_of(uint64_t E, uint32_t m) {
    uint32_t L = 1u;  // bit i of E: bits i .. i+L-1 of the original all set
    while (2u * L <= m) {
        E &= E >> L;
        L *= 2u;
    }
    E &= E >> (m - L);
    return (uint32_t)E & 0xFFFFu;
}

// Byte-equality mask of a chunk against the broadcast byte bb (bit k: byte k).
__device__ __forceinline__ uint32_t eq_mask16(const uint4 c, uint32_t bb) {
    return nibble_of(zero_bytes(c.x ^ bb)) | (nibble_of(zero_bytes(c.y ^ bb)) << 4) |
           (nibble_of(zero_bytes(c.z ^ bb)) << 8) | (nibble_of(zero_bytes(c.w ^ bb)) << 12);
}

template <int NW>
__device__ __forceinline__ uint32_t run_starts16(const uint32_t (&R)[NW], uint32_t bb, uint32_t m) {
    static_assert(NW <= 16, "a 64-bit byte mask");
    uint64_t E = 0ull;
#pragma unroll
    for (int k = 0; k < NW; ++k) E |= (uint64_t)nibble_of(zero_bytes(R[k] ^ bb)) << (4 * k);
    return runs_of(E, m);
}

// The 16 bytes from the 16-byte aligned internal position pc, from the
// staged bytes when they cover them, else from global memory (bytes outside
// the text read as 0).
__device__ __forceinline__ uint4 chunk_at(const SearchJob &J, int64_t pc, const StagedText &T) {
    const int64_t o = pc - T.sbase;
    if (T.inside && o >= 0 && o + 16 <= (int64_t)T.span) return *reinterpret_cast<const uint4 *>(T.buf + o);
    const int64_t wa = pc >> 2;
    uint4 c;
    c.x = wa < 0 ? 0u : load_word(J, (uint64_t)wa);
    c.y = wa + 1 < 0 ? 0u : load_word(J, (uint64_t)(wa + 1));
    c.z = wa + 2 < 0 ? 0u : load_word(J, (uint64_t)(wa + 2));
    c.w = wa + 3 < 0 ? 0u : load_word(J, (uint64_t)(wa + 3));
    return c;
}

// Template argument MP of the strided block and 2-bit code variants' kernels
// for a pattern of period 1 (one byte repeated): kernels of their own, so
// that the period-1 test stays out of the ordinary filter loops.
constexpr int kMpRun = 1;

// The period-1 test of the strided block variant for a whole warp (starts
// 16c - 15 .. 16c of each lane's chunk c, m <= 32): every lane takes the
// byte-equality mask of its own chunk, the next chunk's comes from the next
// lane and the previous chunk's from the lane before (lanes 31 and 0 read the
// chunks past the step), so each chunk's bytes are compared once.  t0: the
// lane's block is marked (a chunk without a marked block has no occurrence).
__device__ __forceinline__ uint32_t run_block16(const SearchJob &J, const uint4 cur, int64_t p0,
                                             const StagedText &T, uint32_t t0, int lane) {
    const uint32_t bb = bcast_byte(J.pat.w[0], 0);
    const uint32_t e_own = eq_mask16(cur, bb);
    uint32_t e_next = __shfl_down_sync(kFull, e_own, 1);
    uint32_t e_prev = __shfl_up_sync(kFull, e_own, 1);
    // lanes 0 and 31 read the chunk before and the chunk after the step in
    // one code path (p0 + 15 is the lane's chunk start, 16-byte aligned)
    if (lane == 0 || lane == 31) {
        const uint32_t e_edge = eq_mask16(chunk_at(J, lane == 0 ? p0 - 1 : p0 + 31, T), bb);
        if (lane == 0) e_prev = e_edge; else e_next = e_edge;
    }
    // bit k of E: byte p0 - 1 + k; start p0 + i is bit i of E >> 1
    const uint64_t E = (uint64_t)e_prev | ((uint64_t)e_own << 16) | ((uint64_t)e_next << 32);
    return t0 ? runs_of(E >> 1, J.pat.m) : 0u;
}

// run_starts16 on the text from p0 (any alignment; m <= 32): 12 words from
// the staged bytes when they cover them, else from global memory (bytes
// outside the text read as 0; the starts they reach are masked by the caller).
__device__ __noinline__ uint32_t run_starts_staged(const SearchJob &J, int64_t p0, const StagedText &T) {
    const int64_t wa = p0 >> 2;  // (floor: p0 may be negative at the text's start)
    const uint32_t sh = (uint32_t)(p0 & 3) * 8u;
    uint32_t W[13];
    const int64_t o = wa * 4 - T.sbase;
    if (T.inside && o >= 0 && o + 52 <= (int64_t)T.span) {
        const uint32_t *S = reinterpret_cast<const uint32_t *>(T.buf) + (o >> 2);
#pragma unroll
        for (int k = 0; k < 13; ++k) W[k] = S[k];
    } else {
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            const int64_t wk = wa + k;
            W[k] = wk < 0 ? 0u : load_word(J, (uint64_t)wk);
        }
    }
    uint32_t R[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) R[k] = __funnelshift_r(W[k], W[k + 1], sh);
    return run_starts16<12>(R, bcast_byte(J.pat.w[0], 0), J.pat.m);
}

// Candidates of the block variant: the chunk's two blocks (those whose
// fingerprint slot is marked: t0, t1) compared with the pattern blocks
// p[j..j+7]; a block match at j gives the candidate 8b - j (Section 3.4).
__device__ __forceinline__ uint32_t block_cands8(const uint4 cur, const uint32_t *pblk, uint32_t t0,
                                                 uint32_t t1) {
    uint32_t cand = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t lo = pblk[2 * j], hi = pblk[2 * j + 1];
        if (t0 && cur.x == lo && cur.y == hi) cand |= 1u << (7 - j);
        if (t1 && cur.z == lo && cur.w == hi) cand |= 1u << (15 - j);
    }
    return kSoundness ? 0xFFFFu : cand;  // soundness build: no block compare either
}

// Candidates of the strided block variant: the chunk's first block against
// p[j..j+7], j < 16, giving the candidate 16c - j (bit 15 - j).
__device__ __forceinline__ uint32_t block_cands16(const uint4 cur, const uint32_t *pblk) {
    uint32_t cand = 0u;
#pragma unroll
    for (int j = 0; j < 16; ++j)
        if (cur.x == pblk[2 * j] && cur.y == pblk[2 * j + 1]) cand |= 1u << (15 - j);
    return kSoundness ? 0xFFFFu : cand;
}

// Full check of one lane's candidates (bit i <-> start p0 + i), in increasing
// order; a candidate that lies q (the pattern's period) after a confirmed
// occurrence needs only its last 8 bytes compared.
__device__ __forceinline__ uint32_t verify_cands_serial(const SearchJob &J, int64_t p0, uint32_t cand,
                                                        const StagedText &T) {
    uint32_t h = 0u;
    int last = -64;
    const int q = (int)J.pat.q;
    while (cand) {
        const int i = __ffs(cand) - 1;
        cand &= cand - 1u;
        const int64_t P = p0 + i;
        if (P < (int64_t)J.delta || P > J.pmax) continue;
        const bool ok = (q != 0 && i - last == q)
                            ? tail8_ok(J, P, T)
                            : verify_staged(J, P, T) &&
                                  (T.mtail == 0u || verify_tail(J, P + 32, T.tail, T.mtail));
        if (ok) {
            h |= 1u << i;
            last = i;
        }
    }
    return h;
}

// Position of the e-th set bit (e = 0, 1, ..) of a 16-bit mask that has more
// than e set bits.
__device__ __forceinline__ uint32_t nth_set_bit16(uint32_t x, uint32_t e) {
    uint32_t pos = 0u, c = __popc(x & 0xFFu);
    if (e >= c) { e -= c; x >>= 8; pos += 8u; }
    c = __popc(x & 0xFu);
    if (e >= c) { e -= c; x >>= 4; pos += 4u; }
    c = __popc(x & 0x3u);
    if (e >= c) { e -= c; x >>= 2; pos += 2u; }
    if (e >= (x & 1u)) pos += 1u;
    return pos;
}

// Warp-cooperative full check of the lanes' candidates (bit i of `cand` <->
// start p0 + i; a whole warp calls it).  The warp's candidates are numbered
// in lane order and each round the 32 lanes check 32 of them, so that a lane
// with many candidates (a run of one byte, a periodic stretch of text) does
// not hold the warp for up to 16 serial checks.  Each check's result goes back
// to the candidate's lane by an OR-reduction over the lanes that checked that
// lane's candidates.  Returns the lane's hits.
__device__ __noinline__ uint32_t coop_verify(const SearchJob &J, int64_t p0, uint32_t cand,
                                             const uint8_t *buf, int64_t sbase, uint32_t inside,
                                             const uint8_t *tail, uint32_t mtail) {
    StagedText T;
    T.buf = buf;
    T.sbase = sbase;
    T.span = (uint32_t)((1024 + 1) * 16);
    T.inside = inside;
    T.tail = tail;
    T.mtail = mtail;
    const int lane = (int)(threadIdx.x & 31u);
    const uint32_t c = __popc(cand);
    const uint32_t incl = warp_incl_scan(c, lane);
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - c;
    uint32_t h = 0u;
    for (uint32_t base = 0; base < total; base += 32u) {
        const uint32_t k = base + (uint32_t)lane;
        // owner of candidate k: the number of lanes whose inclusive count is <= k
        uint32_t L = 0u;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const uint32_t v = __shfl_sync(kFull, incl, (int)(L + (uint32_t)d - 1u));
            if (v <= k) L += (uint32_t)d;
        }
        const bool act = k < total;
        const int src = act ? (int)L : lane;
        const uint32_t cL = __shfl_sync(kFull, cand, src);
        const uint32_t eL = __shfl_sync(kFull, excl, src);
        const int64_t pL = __shfl_sync(kFull, p0, src);
        uint32_t bitv = 0u;
        if (act) {
            const uint32_t bit = nth_set_bit16(cL, k - eL);
            const int64_t P = pL + (int64_t)bit;
            if (P >= (int64_t)J.delta && P <= J.pmax && verify_staged(J, P, T) &&
                (T.mtail == 0u || verify_tail(J, P + 32, T.tail, T.mtail)))
                bitv = 1u << bit;
        }
        // OR of the results over the lanes that checked the same owner's
        // candidates (inactive lanes form their own group)
        const uint32_t grp = __match_any_sync(kFull, act ? L : 32u + (uint32_t)lane);
        const uint32_t orv = __reduce_or_sync(grp, bitv);
        // the owner takes it from the first lane that checked its candidates
        const uint32_t lo = excl > base ? excl : base;
        const uint32_t hi = incl < base + 32u ? incl : base + 32u;
        const uint32_t got = __shfl_sync(kFull, orv, lo < hi ? (int)(lo - base) : lane);
        if (lo < hi) h |= got;
    }
    return h;
}

// Slow path of the block variants, out of line and reached by the whole warp
// when some lane's block hit a marked fingerprint slot (t0: the chunk's first
// block, t1: its second; the strided variant inspects the first only): the
// lanes' candidates from the block compare, checked cooperatively when some
// lane has more than a few, else each lane its own (usually one).
constexpr int kCoopMin = 2;
template <int V>
__device__ __noinline__ uint32_t block_slow(const SearchJob &J, const uint4 cur, int64_t p0,
                                            const uint32_t *pblk, uint32_t t0, uint32_t t1,
                                            const uint8_t *buf, int64_t sbase, uint32_t inside,
                                            const uint8_t *tail, uint32_t mtail) {
    const uint32_t cand = V == V_BLOCK8S ? (t0 ? block_cands16(cur, pblk) : 0u)
                                         : ((t0 | t1) ? block_cands8(cur, pblk, t0, t1) : 0u);
    if (J.pat.q == 1u && J.pat.m <= 32u) {
        // one byte repeated: the chunk's starts decided at once from the text
        if (!cand) return 0u;
        StagedText T;
        T.buf = buf;
        T.sbase = sbase;
        T.span = (uint32_t)((1024 + 1) * 16);
        T.inside = inside;
        T.tail = tail;
        T.mtail = mtail;
        return run_starts_staged(J, p0, T) & cand;
    }
    if (__any_sync(kFull, __popc(cand) > kCoopMin))
        return coop_verify(J, p0, cand, buf, sbase, inside, tail, mtail);
    if (!cand) return 0u;
    StagedText T;
    T.buf = buf;
    T.sbase = sbase;
    T.span = (uint32_t)((1024 + 1) * 16);
    T.inside = inside;
    T.tail = tail;
    T.mtail = mtail;
    return verify_cands_serial(J, p0, cand, T);
}

// Full in-register check of the start at byte 4K + b of the chunk (RR: the
// chunk's words and the next chunk's; m <= 16).
template <int K>
__device__ __forceinline__ bool verify_all_regs(const uint32_t (&RR)[8], uint32_t b, const Pattern &pat) {
    const uint32_t m = pat.m;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if ((uint32_t)(4 * i) < m) {
            const uint32_t win = __funnelshift_r(RR[K + i], RR[K + i + 1], 8u * b);
            ok &= ((win ^ pat.w[i]) & word_mask(m, (uint32_t)i)) == 0u;
        }
    }
    return ok;
}

// Full in-register check of the candidate starts `cand` (bits 0..15) of a
// chunk, given the chunk's words and the next chunk's (m <= 16).
__device__ __noinline__ uint32_t verify_cands_regs(const Pattern &pat, const uint4 cur, uint32_t n0,
                                                   uint32_t n1, uint32_t n2, uint32_t n3,
                                                   uint32_t cand) {
    const uint32_t RR[8] = {cur.x, cur.y, cur.z, cur.w, n0, n1, n2, n3};
    uint32_t h = 0u;
    while (cand) {
        const uint32_t i = (uint32_t)(__ffs(cand) - 1);
        cand &= cand - 1u;
        bool ok;
        switch (i >> 2) {
            case 0: ok = verify_all_regs<0>(RR, i & 3u, pat); break;
            case 1: ok = verify_all_regs<1>(RR, i & 3u, pat); break;
            case 2: ok = verify_all_regs<2>(RR, i & 3u, pat); break;
            default: ok = verify_all_regs<3>(RR, i & 3u, pat); break;
        }
        if (ok) h |= 1u << i;
    }
    return h;
}

// 2-bit code variant (m <= 16): every byte is reduced to its bits 1 and 2
// (a code that tells A, C, G and T apart, upper or lower case), so the 16
// bytes of a chunk give one 32-bit code word, char i at bits 2i..2i+1.  One
// multiply gathers the four codes of a word into its top byte (the partial
// products land on disjoint bits, so no carries), three byte permutes
// assemble the chunk's word.
__device__ __forceinline__ uint32_t code2_of(const uint4 c) {
    // (c & 0x06..) * 0x00820820 == ((c >> 1) & 0x03..) * 0x01041040
    const uint32_t px = (c.x & 0x06060606u) * 0x00820820u;
    const uint32_t py = (c.y & 0x06060606u) * 0x00820820u;
    const uint32_t pz = (c.z & 0x06060606u) * 0x00820820u;
    const uint32_t pw = (c.w & 0x06060606u) * 0x00820820u;
    const uint32_t lo = __byte_perm(px, py, 0x0073u);  // bytes 0, 1: px.b3, py.b3
    const uint32_t hi = __byte_perm(pz, pw, 0x7300u);  // bytes 2, 3: pz.b3, pw.b3
    return __byte_perm(lo, hi, 0x7610u);
}

// Bits 0, 2, .., 30 of z gathered into bits 0..15.
__device__ __forceinline__ uint32_t even_bits(uint32_t z) {
    z = (z | (z >> 1)) & 0x33333333u;
    z = (z | (z >> 2)) & 0x0F0F0F0Fu;
    z = (z | (z >> 4)) & 0x00FF00FFu;
    return (z | (z >> 8)) & 0x0000FFFFu;
}

// 4-byte block variant, slow path: a word k of the chunk (k = 0..3) or the
// next chunk's first word (k = 4) equals a pattern block p[j..j+3] (q[j]); the
// match gives the candidate start 4k - j when it lies in the chunk
// (0 <= 4k - j <= 15), which is then checked in full in registers.
__device__ __noinline__ uint32_t block4_candidates(const Pattern &pat, const uint4 cur, uint32_t n0,
                                                   uint32_t n1, uint32_t n2, uint32_t n3,
                                                   uint32_t q0, uint32_t q1, uint32_t q2, uint32_t q3) {
    const uint32_t R[5] = {cur.x, cur.y, cur.z, cur.w, n0};
    const uint32_t q[4] = {q0, q1, q2, q3};
    uint32_t cand = 0u;
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (4 * k - j >= 0 && 4 * k - j <= 15 && R[k] == q[j]) cand |= 1u << (4 * k - j);
    return verify_cands_regs(pat, cur, n0, n1, n2, n3, cand);
}

// The four pattern blocks p[j..j+3], j = 0..3, of the 4-byte block variant.
__device__ __forceinline__ void pattern_blocks4(const Pattern &pat, uint32_t &q0, uint32_t &q1,
                                                uint32_t &q2, uint32_t &q3) {
    q0 = pat.w[0];
    q1 = __funnelshift_r(pat.w[0], pat.w[1], 8);
    q2 = __funnelshift_r(pat.w[0], pat.w[1], 16);
    q3 = __funnelshift_r(pat.w[0], pat.w[1], 24);
}

// Block test of the 4-byte block variant: does some word of the chunk (or the
// next chunk's first word) equal a pattern block at an offset that gives a
// start inside the chunk?
__device__ __forceinline__ bool block4_any(const uint4 cur, uint32_t n0, uint32_t q0, uint32_t q1,
                                           uint32_t q2, uint32_t q3) {
    return (cur.x == q0) | (cur.y == q0) | (cur.y == q1) | (cur.y == q2) | (cur.y == q3) |
           (cur.z == q0) | (cur.z == q1) | (cur.z == q2) | (cur.z == q3) | (cur.w == q0) |
           (cur.w == q1) | (cur.w == q2) | (cur.w == q3) | (n0 == q1) | (n0 == q2) | (n0 == q3);
}

// The 16 byte flags of four zero_bytes() words (bit 7 of each byte) as a
// 16-bit mask, bit 4k + b for byte b of word k.  Words k and k + 1 share one
// 32 x 32 -> 64-bit multiply: with word k's flags moved to bits 8b and word
// k + 1's to bits 8b + 4, the constant's term 2^(28 - 7b) carries byte b's two
// flags to bits 28 + b and 32 + b, and no two partial products meet, so the
// product's bits 28..35 are the two words' nibbles (half the shifts and ORs
// of packing each word alone, and the multiplies run on the FMA pipe).
__device__ __forceinline__ uint32_t pack_flags4(uint32_t z0, uint32_t z1, uint32_t z2, uint32_t z3) {
    const uint64_t a = (uint64_t)((z0 >> 7) | (z1 >> 3)) * 0x10204080ull;
    const uint64_t b = (uint64_t)((z2 >> 7) | (z3 >> 3)) * 0x10204080ull;
    return ((uint32_t)(a >> 28) & 0xFFu) | (((uint32_t)(b >> 28) & 0xFFu) << 8);
}

// Hit mask of one chunk (before start-validity masking).
//   cur    the chunk's words; nsrc: this lane's contribution to the neighbour
//   shuffle (the chunk the lane before needs as "next chunk").
template <int V, int MP>
__device__ __forceinline__ uint32_t chunk_hits(const SearchJob &J, const uint4 cur,
                                               const uint4 nsrc, int64_t p0,
                                               const BcastWords &B, const uint32_t *table,
                                               const uint32_t *pblk, int lane,
                                               const StagedText &T) {
    const int src = (lane + 1) & 31;
    const Pattern &pat = J.pat;
    if constexpr (V == V_DIRECT) {
        // Section 3.2 (EPSMa): every start is compared against the whole
        // (m <= 4) pattern at once; no verify step.
        // MP = 0: m read at run time (one code path for m = 1..4); the
        // compares of bytes at or past m are masked off.
        uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
        uint32_t R[5] = {cur.x, cur.y, cur.z, cur.w, n0};
        const uint32_t mk1 = (MP == 0 && pat.m <= 1u) ? 0u : 0xFFFFFFFFu;
        const uint32_t mk2 = (MP == 0 && pat.m <= 2u) ? 0u : 0xFFFFFFFFu;
        const uint32_t mk3 = (MP == 0 && pat.m <= 3u) ? 0u : 0xFFFFFFFFu;
        uint32_t z[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t X;
            if constexpr (MP == 0) {
                X = (R[k] ^ B.b[0]) | ((__funnelshift_r(R[k], R[k + 1], 8) ^ B.b[1]) & mk1) |
                    ((__funnelshift_r(R[k], R[k + 1], 16) ^ B.b[2]) & mk2) |
                    ((__funnelshift_r(R[k], R[k + 1], 24) ^ B.b[3]) & mk3);
            } else {
                X = window_mismatch<MP>(0u, R[k], R[k + 1], B.b[0], B.b[1], B.b[2], B.b[3]);
            }
            z[k] = zero_bytes(X);
        }
        // most chunks of a large alphabet have no match: skip the packing
        if ((z[0] | z[1] | z[2] | z[3]) == 0u) return 0u;
        return pack_flags4(z[0], z[1], z[2], z[3]);
    } else if constexpr (kSoundness && (V == V_PREFIX4 || V == V_PREFIX8 || V == V_BLOCK4)) {
        // soundness build: every start is a candidate, checked in full
        const uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
        const uint32_t n1 = __shfl_sync(kFull, nsrc.y, src);
        const uint32_t n2 = __shfl_sync(kFull, nsrc.z, src);
        const uint32_t n3 = __shfl_sync(kFull, nsrc.w, src);
        return verify_cands_regs(pat, cur, n0, n1, n2, n3, 0xFFFFu);
    } else if constexpr (V == V_PREFIX4) {
        // Section 3.3 (EPSMb) with a 4-byte prefix: exact prefix test per start,
        // then the remaining bytes are checked in registers.
        uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
        uint32_t R[5] = {cur.x, cur.y, cur.z, cur.w, n0};
        uint32_t X[4];
        uint32_t any = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            X[k] = window_mismatch<4>(0u, R[k], R[k + 1], B.b[0], B.b[1], B.b[2], B.b[3]);
            any |= has_zero_byte(X[k]);
        }
        uint32_t h = 0u;
        if (__any_sync(kFull, any != 0u)) {
            uint32_t n1 = __shfl_sync(kFull, nsrc.y, src);
            uint32_t n2 = __shfl_sync(kFull, nsrc.z, src);
            uint32_t n3 = __shfl_sync(kFull, nsrc.w, src);
            const uint32_t RR[8] = {cur.x, cur.y, cur.z, cur.w, n0, n1, n2, n3};
            if (any) {
                h |= verify_word_hits<0>(zero_bytes(X[0]), RR, 1u, pat);
                h |= verify_word_hits<1>(zero_bytes(X[1]), RR, 1u, pat);
                h |= verify_word_hits<2>(zero_bytes(X[2]), RR, 1u, pat);
                h |= verify_word_hits<3>(zero_bytes(X[3]), RR, 1u, pat);
            }
        }
        return h;
    } else if constexpr (V == V_PREFIX8) {
        // Section 3.3 (EPSMb) with the paper's m' = 8 prefix: the prefix
        // mismatch at start 4k+b is byte b of X_k | Y_{k+1}, X for p[0..3] at
        // word k and Y for p[4..7] at word k+1.
        uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
        uint32_t n1 = __shfl_sync(kFull, nsrc.y, src);
        uint32_t R[6] = {cur.x, cur.y, cur.z, cur.w, n0, n1};
        uint32_t Z[4];
        uint32_t any = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t X = window_mismatch<4>(0u, R[k], R[k + 1], B.b[0], B.b[1], B.b[2], B.b[3]);
            Z[k] = window_mismatch<4>(X, R[k + 1], R[k + 2], B.b[4], B.b[5], B.b[6], B.b[7]);
            any |= has_zero_byte(Z[k]);
        }
        uint32_t h = 0u;
        if (__any_sync(kFull, any != 0u)) {
            uint32_t n2 = __shfl_sync(kFull, nsrc.z, src);
            uint32_t n3 = __shfl_sync(kFull, nsrc.w, src);
            const uint32_t RR[8] = {cur.x, cur.y, cur.z, cur.w, n0, n1, n2, n3};
            if (any) {
                h |= verify_word_hits<0>(zero_bytes(Z[0]), RR, 2u, pat);
                h |= verify_word_hits<1>(zero_bytes(Z[1]), RR, 2u, pat);
                h |= verify_word_hits<2>(zero_bytes(Z[2]), RR, 2u, pat);
                h |= verify_word_hits<3>(zero_bytes(Z[3]), RR, 2u, pat);
            }
        }
        return h;
    } else if constexpr (V == V_BLOCK4) {
        // Section 3.4's aligned-block idea with 4-byte blocks (7 <= m <= 16):
        // every occurrence at s covers the aligned word at the first multiple
        // of 4 in [s, s+3], equal to the pattern block p[j..j+3] with j that
        // word's offset from s -- only four blocks, so each word is compared
        // with all of them instead of hashing.
        const uint32_t n0 = __shfl_sync(kFull, nsrc.x, src);
        uint32_t q0, q1, q2, q3;
        pattern_blocks4(pat, q0, q1, q2, q3);
        const bool any = block4_any(cur, n0, q0, q1, q2, q3);
        uint32_t h = 0u;
        if (__any_sync(kFull, any)) {
            const uint32_t n1 = __shfl_sync(kFull, nsrc.y, src);
            const uint32_t n2 = __shfl_sync(kFull, nsrc.z, src);
            const uint32_t n3 = __shfl_sync(kFull, nsrc.w, src);
            if (any) h = block4_candidates(pat, cur, n0, n1, n2, n3, q0, q1, q2, q3);
        }
        return h;
    } else if constexpr (V == V_BLOCK8S) {
        // Section 3.4 (EPSMc) with the block stride sh of two blocks: only
        // the chunk's first block is fingerprinted (half the hashing and
        // lookups of the plain block variant); starts 16c - 15 .. 16c.
        const uint32_t t0 = kSoundness ? 1u : table_bit(table, block_hash(cur.x, cur.y, pat.kbits));
        if (!__any_sync(kFull, t0 != 0u)) return 0u;
        if constexpr (MP == kMpRun) return run_block16(J, cur, p0, T, t0, lane);
        return block_slow<V_BLOCK8S>(J, cur, p0, pblk, t0, 0u, T.buf, T.sbase, T.inside, T.tail,
                                     T.mtail);
    } else {
        // Section 3.4 (EPSMc) on aligned 8-byte blocks: fingerprint each block,
        // and where the slot is marked compare the block with the pattern
        // blocks p[j..j+7]; a block match at j gives the candidate 8b - j,
        // which is then checked in full.
        const uint32_t t0 = kSoundness ? 1u : table_bit(table, block_hash(cur.x, cur.y, pat.kbits));
        const uint32_t t1 = kSoundness ? 1u : table_bit(table, block_hash(cur.z, cur.w, pat.kbits));
        if (!__any_sync(kFull, (t0 | t1) != 0u)) return 0u;
        return block_slow<V_BLOCK8>(J, cur, p0, pblk, t0, t1, T.buf, T.sbase, T.inside, T.tail,
                                    T.mtail);
    }
}

}  // namespace epsm
