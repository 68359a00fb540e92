/* Test driver: runs the oracle's DT and RS dynamics, sums and power sums on a
 * few small lattices so the oracle can be built and exercised under the host
 * address and undefined-behaviour sanitizers.  Prints a checksum. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

typedef struct {
    int32_t L, N, Tx, Ty, phase_order, pad_;
    uint64_t seed;
} orc_params;

int orc_sweeps(const orc_params* P, int64_t* h, const uint32_t* lanes, int32_t n_lanes, uint64_t t0,
               uint64_t n_sweeps, int32_t rs, int32_t n_threads, int64_t* accepted);
void orc_sums(const int64_t* h, int32_t L, int32_t n_lanes, int64_t* sum_h, int64_t* sum_h2_hi, uint64_t* sum_h2_lo);
void orc_power_sums(const int64_t* h, int32_t L, int32_t n_lanes, int64_t* out);
void orc_max_step(const int64_t* h, int32_t L, int32_t n_lanes, int64_t* out);

int main(void)
{
    const int32_t cases[][5] = {{8, 1, 2, 2, 0}, {16, 2, 4, 4, 1}, {24, 7, 8, 8, 0}, {32, 3, 16, 16, 0}, {6, 1, 2, 2, 0}};
    uint64_t check = 0;
    for (unsigned c = 0; c < sizeof(cases) / sizeof(cases[0]); ++c) {
        for (int rs = 0; rs < 2; ++rs) {
            orc_params P = {cases[c][0], cases[c][1], cases[c][2], cases[c][3], cases[c][4], 0, 1234u + c};
            const int32_t L = P.L, n = 3;
            int64_t* h = calloc((size_t)n * L * L, sizeof(int64_t));
            uint32_t lanes[3] = {0, 5, 31};
            int64_t acc[3] = {0, 0, 0};
            if (!h || orc_sweeps(&P, h, lanes, n, 0, 20, rs, 2, acc) != 0) return 1;
            int64_t s1[3], hi[3], ps[24], mx[3];
            uint64_t lo[3];
            orc_sums(h, L, n, s1, hi, lo);
            orc_power_sums(h, L, n, ps);
            orc_max_step(h, L, n, mx);
            for (int j = 0; j < n; ++j) {
                if (mx[j] > P.N) return 2;                      /* constraint of Eq. 6 */
                if (ps[8 * j] != s1[j] || acc[j] != s1[j]) return 3;  /* sum h = deposits */
                check = check * 31u + (uint64_t)s1[j] + lo[j];
            }
            free(h);
        }
    }
    printf("%llu\n", (unsigned long long)check);
    return 0;
}
