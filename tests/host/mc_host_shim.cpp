// Host build of the device marching-cubes routine (csrc/mcubes.cuh), so that a
// CPU test can compare its triangles with the FP64 oracle's bit for bit.
// Compiled by the test with -ffp-contract=off.
#include "../../paper_2101_12408_gb300/csrc/mcubes.cuh"

extern "C" int mc_host_cube(const double* cphi, const int* q, double dx, double* out) {
    const double origin[3] = {0.0, 0.0, 0.0};
    return mpm::mc::cube_triangles(cphi, q, dx, origin,
                                   [&](int t, const double* p0, const double* p1, const double* p2) {
                                       for (int a = 0; a < 3; ++a) {
                                           out[t * 9 + a] = p0[a];
                                           out[t * 9 + 3 + a] = p1[a];
                                           out[t * 9 + 6 + a] = p2[a];
                                       }
                                   });
}
