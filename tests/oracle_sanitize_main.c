/*
 * oracle_sanitize_main.c -- test driver that runs the oracle (fec_oracle.c)
 * under the host address and undefined-behaviour sanitizers.
 *
 * Built by tests/test_oracle_sanitize.py together with ../oracle/fec_oracle.c
 * and -fsanitize=address,undefined -fno-sanitize-recover=all, so any invalid
 * access, leak, overflow of a signed type or misaligned access aborts the
 * process with a report.
 *
 * Input file (little-endian, written by the Python test from the seeded
 * generators): a sequence of cases, each
 *     int64 n, float d, int64 min_size, int64 max_size, int32 brute,
 *     float xyz[3n]
 * For every case it runs fec_oracle_cluster (kd-tree BFS) and, when brute is
 * set, fec_oracle_bruteforce (all pairs), and prints one line:
 *     <status> <num_clusters> <fnv1a-64 of the labels> [<brute status> <equal>]
 * The Python test compares these lines with the oracle run unsanitized.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int fec_oracle_cluster(const float *xyz, int64_t n, float d, int64_t min_size,
                       int64_t max_size, int32_t *labels, int32_t *num_clusters);
int fec_oracle_bruteforce(const float *xyz, int64_t n, float d, int64_t min_size,
                          int64_t max_size, int32_t *labels, int32_t *num_clusters);

static uint64_t fnv1a(const int32_t *v, int64_t n)
{
    uint64_t h = 1469598103934665603ull;
    const unsigned char *b = (const unsigned char *)v;
    for (int64_t i = 0; i < n * 4; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

int main(int argc, char **argv)
{
    if (argc != 2) {
        fprintf(stderr, "usage: %s cases.bin\n", argv[0]);
        return 2;
    }
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    for (;;) {
        int64_t n, mn, mx;
        float d;
        int32_t brute;
        if (fread(&n, 8, 1, f) != 1) break;
        if (fread(&d, 4, 1, f) != 1 || fread(&mn, 8, 1, f) != 1 || fread(&mx, 8, 1, f) != 1 ||
            fread(&brute, 4, 1, f) != 1 || n < 0) {
            fclose(f);
            return 3;
        }
        /* exact-size allocations, so that the address sanitizer sees any
         * access one past the end */
        float *xyz = (float *)malloc(n > 0 ? (size_t)n * 12 : 1);
        int32_t *lab = (int32_t *)malloc(n > 0 ? (size_t)n * 4 : 1);
        int32_t *lab2 = (int32_t *)malloc(n > 0 ? (size_t)n * 4 : 1);
        if (!xyz || !lab || !lab2 || (n > 0 && fread(xyz, 12, (size_t)n, f) != (size_t)n)) {
            fclose(f);
            return 3;
        }
        int32_t k = -1, k2 = -1;
        const int st = fec_oracle_cluster(xyz, n, d, mn, mx, lab, &k);
        printf("%d %d %016llx", st, (int)k,
               (unsigned long long)(st == 0 ? fnv1a(lab, n) : 0ull));
        if (brute) {
            const int st2 = fec_oracle_bruteforce(xyz, n, d, mn, mx, lab2, &k2);
            const int same = st2 == st && (st != 0 || (k2 == k && memcmp(lab, lab2, (size_t)n * 4) == 0));
            printf(" %d %d", st2, same);
        }
        printf("\n");
        free(xyz);
        free(lab);
        free(lab2);
    }
    fclose(f);
    return 0;
}
