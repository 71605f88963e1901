// Device side of the seeded input generators (see textgen.h): fills device
// buffers with the same bytes gen_host.c produces.  No string-matching
// arithmetic lives here; it only makes synthetic inputs in HBM.
#include <cuda_runtime.h>
#include <stdint.h>
#include "textgen.h"

#define GEN_API extern "C" __attribute__((visibility("default")))

// Each thread makes 16 consecutive bytes (4 draws) and stores them as one
// 16-byte vector when the destination allows it.
__global__ void gen_iid_kernel(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                               const uint8_t *__restrict__ table) {
    uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16ULL;
    for (; i0 < len; i0 += (uint64_t)gridDim.x * blockDim.x * 16ULL) {
        uint8_t b[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) b[k] = gen_iid_byte(key, start + i0 + k, table);
        if (i0 + 16 <= len && ((reinterpret_cast<uintptr_t>(dst + i0) & 15) == 0)) {
            uint4 v;
            v.x = b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24);
            v.y = b[4] | (b[5] << 8) | (b[6] << 16) | ((uint32_t)b[7] << 24);
            v.z = b[8] | (b[9] << 8) | (b[10] << 16) | ((uint32_t)b[11] << 24);
            v.w = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
            *reinterpret_cast<uint4 *>(dst + i0) = v;
        } else {
            for (int k = 0; k < 16 && i0 + k < len; ++k) dst[i0 + k] = b[k];
        }
    }
}

// One thread per Markov segment overlapping [start, start+len).
__global__ void gen_markov_kernel(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                                  const uint8_t *start_table, const uint8_t *rows,
                                  const uint8_t *sym_index, uint64_t seg0, uint64_t nseg) {
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nseg) return;
    uint64_t seg = seg0 + k;
    uint64_t seg_base = seg * GEN_MARKOV_SEG;
    uint64_t end = start + len;
    uint64_t lo = seg_base > start ? seg_base : start;
    uint64_t hi = seg_base + GEN_MARKOV_SEG < end ? seg_base + GEN_MARKOV_SEG : end;
    if (lo >= hi) return;
    gen_markov_segment(key, seg, lo - seg_base, hi - seg_base, start_table, rows, sym_index,
                       dst + (lo - start));
}

__global__ void gen_runs_kernel(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                                uint64_t block, uint32_t maxlen, uint8_t run_byte) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (gen_in_run(key, start + i, block, maxlen)) dst[i] = run_byte;
}

static int grid_for(uint64_t work, int threads) {
    uint64_t g = (work + threads - 1) / threads;
    if (g > 152ULL * 64ULL) g = 152ULL * 64ULL;
    if (g < 1) g = 1;
    return (int)g;
}

GEN_API int gen_fill_iid_device(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                                const uint8_t *table_dev, void *stream) {
    if (len == 0) return 0;
    gen_iid_kernel<<<grid_for((len + 15) / 16, 256), 256, 0, (cudaStream_t)stream>>>(
        dst, start, len, key, table_dev);
    return (int)cudaGetLastError();
}

GEN_API int gen_fill_markov_device(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                                   const uint8_t *start_table_dev, const uint8_t *rows_dev,
                                   const uint8_t *sym_index_dev, void *stream) {
    if (len == 0) return 0;
    uint64_t seg0 = start / GEN_MARKOV_SEG;
    uint64_t seg1 = (start + len - 1) / GEN_MARKOV_SEG;
    uint64_t nseg = seg1 - seg0 + 1;
    int threads = 128;
    gen_markov_kernel<<<(unsigned)((nseg + threads - 1) / threads), threads, 0,
                        (cudaStream_t)stream>>>(dst, start, len, key, start_table_dev, rows_dev,
                                                sym_index_dev, seg0, nseg);
    return (int)cudaGetLastError();
}

GEN_API int gen_apply_runs_device(uint8_t *dst, uint64_t start, uint64_t len, uint64_t key,
                                  uint64_t block, uint32_t maxlen, uint8_t run_byte,
                                  void *stream) {
    if (len == 0) return 0;
    gen_runs_kernel<<<grid_for(len, 256), 256, 0, (cudaStream_t)stream>>>(
        dst, start, len, key, block, maxlen, run_byte);
    return (int)cudaGetLastError();
}
