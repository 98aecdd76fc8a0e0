/*
 * ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU statement of what the GPU sorter computes.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it; the sorting
 * library never does.  It shares no code, header or table with the GPU path.
 *
 * What is computed (Kokot, Deorowicz, Dlugosz, "Even faster sorting of (not only)
 * integers", section 1): sorting n records by a key.  A record is rec_size bytes; its key
 * is the first key_size bytes read as a little-endian unsigned integer (byte key_size-1 is
 * the most significant); the other bytes are data that travels with the key.
 *
 * The sort is the LSD radix sort described in section 1: one phase per key digit, from the
 * least significant digit to the most significant, each phase a stable counting sort
 * (count the digit values, turn the counts into starting offsets by an exclusive prefix
 * sum, move every record to the next free slot of its digit value in input order).  The
 * digits of the full sort are the key bytes (the paper's 1-byte digits, section 3.1).
 *
 * Since every phase is stable, the result is the unique stable sort by key: keys are
 * non-decreasing and records with equal keys keep their input order.
 *
 * oracle_partition_bits() is one such phase on an arbitrary digit (a contiguous range of
 * key bits); it is what one distribution pass of an MSD radix sort computes on its bin
 * (section 1, the first step of section 3.1), so the GPU's passes can be checked alone.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Value of key bits [lo, lo + width) of one record; key bit b is bit (b mod 8) of key
 * byte floor(b / 8).  Requires lo + width <= 8 * key_size and width <= 24. */
static uint32_t digit_of(const uint8_t *rec, uint32_t lo, uint32_t width) {
    uint32_t v = 0;
    for (uint32_t j = 0; j < width; j++) {
        uint32_t b = lo + j;
        uint32_t bit = (rec[b >> 3] >> (b & 7)) & 1u;
        v |= bit << j;
    }
    return v;
}

/* One stable counting-sort phase: records of src are moved to dst ordered by the digit
 * made of key bits [lo, lo + width).  Returns 0, or -1 on bad arguments / no memory. */
int oracle_partition_bits(const uint8_t *src, uint8_t *dst, uint64_t n, uint32_t rec_size,
                          uint32_t key_size, uint32_t lo, uint32_t width) {
    if (width == 0 || width > 24 || lo + width > 8u * key_size || key_size > rec_size) return -1;
    uint64_t buckets = 1ull << width;
    uint64_t *count = (uint64_t *)calloc(buckets, sizeof(uint64_t));
    if (!count) return -1;
    /* count */
    for (uint64_t i = 0; i < n; i++) count[digit_of(src + i * rec_size, lo, width)]++;
    /* exclusive prefix sum: count[v] becomes the first slot of digit value v */
    uint64_t run = 0;
    for (uint64_t v = 0; v < buckets; v++) { uint64_t c = count[v]; count[v] = run; run += c; }
    /* stable scatter, in input order */
    for (uint64_t i = 0; i < n; i++) {
        uint32_t v = digit_of(src + i * rec_size, lo, width);
        memcpy(dst + count[v] * rec_size, src + i * rec_size, rec_size);
        count[v]++;
    }
    free(count);
    return 0;
}

/* Histogram of the digit made of key bits [lo, lo + width): counts[v] = number of records
 * whose digit equals v (counts has 2^width entries). */
int oracle_histogram_bits(const uint8_t *src, uint64_t n, uint32_t rec_size, uint32_t key_size,
                          uint32_t lo, uint32_t width, uint64_t *counts) {
    if (width == 0 || width > 24 || lo + width > 8u * key_size || key_size > rec_size) return -1;
    memset(counts, 0, sizeof(uint64_t) << width);
    for (uint64_t i = 0; i < n; i++) counts[digit_of(src + i * rec_size, lo, width)]++;
    return 0;
}

/* LSD radix sort with 1-byte digits, least significant first; the sorted records end in
 * buf (tmp is scratch of the same size).  Returns 0 or -1. */
int oracle_lsd_sort(uint8_t *buf, uint8_t *tmp, uint64_t n, uint32_t rec_size, uint32_t key_size) {
    if (rec_size == 0 || key_size == 0 || key_size > rec_size) return -1;
    uint8_t *src = buf, *dst = tmp;
    for (uint32_t byte = 0; byte < key_size; byte++) {
        if (oracle_partition_bits(src, dst, n, rec_size, key_size, 8 * byte, 8) != 0) return -1;
        uint8_t *t = src; src = dst; dst = t;
    }
    if (src != buf) memcpy(buf, src, n * rec_size);
    return 0;
}

/* Independent sorts of consecutive segments: segment s is records [offsets[s], offsets[s+1]).
 * offsets has n_segs + 1 entries, non-decreasing, offsets[0] = 0. */
int oracle_sort_segmented(uint8_t *buf, uint8_t *tmp, const uint64_t *offsets, uint64_t n_segs,
                          uint32_t rec_size, uint32_t key_size) {
    for (uint64_t s = 0; s < n_segs; s++) {
        uint64_t a = offsets[s], b = offsets[s + 1];
        if (b < a) return -1;
        if (oracle_lsd_sort(buf + a * rec_size, tmp + a * rec_size, b - a, rec_size, key_size) != 0) return -1;
    }
    return 0;
}

/* Run-length count of equal keys (the counting step after the sort in k-mer counting, the
 * paper's application in section 4): a run is a maximal range of consecutive records whose
 * keys (bytes [0, key_size)) are equal.  first receives the first record of every run,
 * counts[r] the number of records in run r; *nruns the number of runs.  Returns 0 or -1. */
int oracle_count_runs(const uint8_t *src, uint64_t n, uint32_t rec_size, uint32_t key_size, uint8_t *first,
                      uint64_t *counts, uint64_t *nruns) {
    if (rec_size == 0 || key_size == 0 || key_size > rec_size) return -1;
    uint64_t r = 0;
    for (uint64_t i = 0; i < n; i++) {
        const uint8_t *rec = src + i * rec_size;
        if (i == 0 || memcmp(rec, rec - rec_size, key_size) != 0) {
            memcpy(first + r * rec_size, rec, rec_size);
            counts[r] = 0;
            r++;
        }
        counts[r - 1]++;
    }
    *nruns = r;
    return 0;
}
