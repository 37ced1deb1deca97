// scaled.cu -- diagonal scalings of the operator: the products and solves of
// A(c) = H diag(c) used by gradients with respect to per-panel density
// coefficients (the single-layer potential of Sec. 2.1 with the density
// u_j = c_j alpha_j on panel j).  Vectors are [nrhs][n] in the caller's
// original panel order, so the scale of entry e is d[e mod n].
#include <algorithm>

#include "hm_internal.cuh"

namespace hm {

static unsigned sgrid(int64_t total) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 8 * (int64_t)num_sms()));
}

// out = a / d (entry-wise, d repeated over the right-hand sides)
__global__ void div_diag_kernel(const double *__restrict__ a, const double *__restrict__ d, int64_t n, int64_t total,
                                double *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = a[e] / d[e % n];
}

// out = d * a (d == nullptr: a copy)
__global__ void mul_diag_kernel(const double *__restrict__ a, const double *__restrict__ d, int64_t n, int64_t total,
                                double *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = d ? d[e % n] * a[e] : a[e];
}

// y = alpha * (d * v) + beta * y (d == nullptr: the identity; beta == 0: y is not read)
__global__ void axpby_diag_kernel(const double *__restrict__ v, const double *__restrict__ d, int64_t n,
                                  int64_t total, double alpha, double beta, double *__restrict__ y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double t = alpha * (d ? d[e % n] * v[e] : v[e]);
        y[e] = beta == 0.0 ? t : t + beta * y[e];
    }
}

void div_diag(const double *a, const double *d, int64_t n, int nrhs, double *out, cudaStream_t s) {
    const int64_t total = n * (int64_t)nrhs;
    div_diag_kernel<<<sgrid(total), 256, 0, s>>>(a, d, n, total, out);
    HM_LAUNCH_CHECK();
}

void mul_diag(const double *a, const double *d, int64_t n, int nrhs, double *out, cudaStream_t s) {
    const int64_t total = n * (int64_t)nrhs;
    mul_diag_kernel<<<sgrid(total), 256, 0, s>>>(a, d, n, total, out);
    HM_LAUNCH_CHECK();
}

void axpby_diag(const double *v, const double *d, int64_t n, int nrhs, double alpha, double beta, double *y,
                cudaStream_t s) {
    const int64_t total = n * (int64_t)nrhs;
    axpby_diag_kernel<<<sgrid(total), 256, 0, s>>>(v, d, n, total, alpha, beta, y);
    HM_LAUNCH_CHECK();
}

}  // namespace hm
