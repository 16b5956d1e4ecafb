// Layout of the FP64 swap tables (Sec. 2.4) shared by the FP64 M2L and M2M
// kernels: the cosine block of degree n, (n+1) x (n+1), starts at cos_off(n);
// the sine block, n x n, at sin_off(n) (both row-major, generated exactly by
// gen_swap.py).
#pragma once

namespace gbfmm {

__host__ __device__ constexpr int cos_off(int n) { return n * (n + 1) * (2 * n + 1) / 6; }
__host__ __device__ constexpr int sin_off(int n) { return (n - 1) * n * (2 * n - 1) / 6; }

struct Swap64 {
    const double* cosb;
    const double* sinb;
};

}  // namespace gbfmm
