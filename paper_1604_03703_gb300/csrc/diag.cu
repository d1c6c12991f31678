// diag.cu -- self-check entry point for the mixed form's Householder
// scalars: evaluates house_scalars_f2 (pair-float) and house_scalars (FP64,
// rounded to FP32) on the same inputs so a test can hold them equal.
#include "common.cuh"

namespace sev {

__global__ void diag_house_kernel(int count, const float *__restrict__ alpha, const float *__restrict__ ssq_hi,
                                  const float *__restrict__ ssq_lo, float *__restrict__ out_f2,
                                  float *__restrict__ out_f64) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        float t, b, v;
        house_scalars_f2(alpha[i], F2{ssq_hi[i], ssq_lo[i]}, &t, &b, &v);
        out_f2[3 * i] = t;
        out_f2[3 * i + 1] = b;
        out_f2[3 * i + 2] = v;
        double td, bd, vd;
        house_scalars((double)alpha[i], (double)ssq_hi[i] + (double)ssq_lo[i], &td, &bd, &vd);
        out_f64[3 * i] = (float)td;
        out_f64[3 * i + 1] = (float)bd;
        out_f64[3 * i + 2] = (float)vd;
    }
}

}  // namespace sev

extern "C" int sev_diag_house_scalars(int count, const float *alpha, const float *ssq_hi, const float *ssq_lo,
                                      float *out_pairfloat, float *out_fp64, void *stream) {
    if (count < 0) return -1;
    if (count == 0) return 0;
    if (!alpha || !ssq_hi || !ssq_lo) return -2;
    if (!out_pairfloat || !out_fp64) return -5;
    int grid = (count + 255) / 256;
    if (grid > 4096) grid = 4096;
    sev::diag_house_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(count, alpha, ssq_hi, ssq_lo, out_pairfloat,
                                                                   out_fp64);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
