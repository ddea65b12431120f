// Test program for fec_cluster_noalloc across a device reset (built and run
// by tests/test_zz_no_alloc.py, linked with the library's own objects so that
// it shares the library's CUDA runtime).
//
// The entry point keeps the device address of its static workspace from its
// set-up step.  That address belongs to the CUDA context it was taken in; after
// cudaDeviceReset the next call runs in a new context, must redo the set-up,
// and must give the same labels as before the reset.  Prints one line and
// exits 0 when both calls return FEC_OK with equal labels and cluster counts.
#include <cstdint>
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#include "fec.h"

int main()
{
    // 40 small clusters of 100 points on a line, 2 m apart (multiples of 1/1024 m),
    // shuffled by a fixed linear congruential sequence.
    const int n = 4000;
    std::vector<float> xyz(3 * n);
    uint32_t s = 12345u;
    auto next = [&]() {
        s = s * 1664525u + 1013904223u;
        return s >> 8;
    };
    for (int i = 0; i < n; ++i) {
        const int c = i / 100;
        xyz[3 * i + 0] = (float)(2048 * c + (int)(next() % 200)) / 1024.0f;
        xyz[3 * i + 1] = (float)(next() % 200) / 1024.0f;
        xyz[3 * i + 2] = (float)(next() % 200) / 1024.0f;
    }
    for (int i = n - 1; i > 0; --i) {
        const int j = (int)(next() % (uint32_t)(i + 1));
        for (int a = 0; a < 3; ++a) {
            const float t = xyz[3 * i + a];
            xyz[3 * i + a] = xyz[3 * j + a];
            xyz[3 * j + a] = t;
        }
    }
    std::vector<int32_t> l1(n, -7), l2(n, -7);
    int32_t k1 = -1, k2 = -1;
    const fec_status s1 =
        fec_cluster_noalloc(xyz.data(), n, 0.3f, 1, INT64_MAX, l1.data(), &k1, nullptr);
    const cudaError_t r = cudaDeviceReset();
    const fec_status s2 =
        fec_cluster_noalloc(xyz.data(), n, 0.3f, 1, INT64_MAX, l2.data(), &k2, nullptr);
    bool same = true;
    for (int i = 0; i < n; ++i) same = same && l1[i] == l2[i];
    std::printf("first %s k=%d, reset %d, second %s k=%d, labels %s\n", fec_status_string(s1), k1,
                (int)r, fec_status_string(s2), k2, same ? "equal" : "differ");
    return (s1 == FEC_OK && r == cudaSuccess && s2 == FEC_OK && k1 == 40 && k1 == k2 && same) ? 0
                                                                                              : 1;
}
