// Compile-only check that the public device header is self-contained: a
// user kernel including nothing else calls both device-callable solvers
// (compiled, not run, by tests/test_device_header.py).
#include "tinylu_device.cuh"
__global__ void k(double *A, double *b, int *p, int *info)
{
    double a[3][3], bb[3];
    int piv[3];
    for (int i = 0; i < 3; ++i) { bb[i] = b[i]; for (int j = 0; j < 3; ++j) a[i][j] = A[3 * j + i]; }
    info[0] = tl::lupp_solve<3>(a, bb, piv);
    double g[2][4], gb[2];
    int gp[2];
    for (int s = 0; s < 2; ++s) { gb[s] = b[s]; for (int j = 0; j < 4; ++j) g[s][j] = A[j + 4 * s]; }
    info[1] = tl::lupp_solve_subwarp<4, 2>(g, gb, gp);
    for (int i = 0; i < 3; ++i) { b[i] = bb[i]; p[i] = piv[i]; }
    for (int s = 0; s < 2; ++s) { b[3 + s] = gb[s]; p[3 + s] = gp[s]; }
}
