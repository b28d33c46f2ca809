// Stable LSD radix sort of (key, value) pairs of 32-bit words, shared by the
// binning and the cache's spatial order (binsort.cu implements it).
#pragma once
#include "common.cuh"

namespace gs3 {

// Words of the digit-count scratch radix_sort_pairs needs.
size_t radix_sort_hist_words();

// Sorts n pairs stably on the low `bits` bits of the key, one byte-digit
// pass each (a pass whose digit is the same for every key is a copy).  The
// pairs start in k[0], v[0]; k[1], v[1] are the second buffers (n words
// each); on return `cur` is the buffer holding the result.  hist: scratch of
// radix_sort_hist_words() words.
gs_status radix_sort_pairs(uint32_t *k[2], uint32_t *v[2], int64_t n, int bits, uint32_t *hist, int &cur,
                           cudaStream_t st);

}  // namespace gs3
