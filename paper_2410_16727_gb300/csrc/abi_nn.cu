// abi_nn.cu -- C ABI of the denoiser layers (kernels in kernels_nn.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dseed {
int set_error(int code, const char *fmt, ...);
int nn_gemm_f32(int ta, int tb, int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb,
                float beta, float *C, int ldc, const float *bias, cudaStream_t st);
int nn_gemm_bf16(int M, int N, int K, const void *A, const void *W, float *C, const float *bias, cudaStream_t st);
int nn_im2col1d(const float *x, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad, void *cols, int bf16,
                cudaStream_t st);
int nn_col2im1d(const float *cols, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad, float *dx,
                cudaStream_t st);
int nn_colsum(const float *y, int R, int C, float *out, int accumulate, cudaStream_t st);
int nn_gn_fwd(const float *x, int N, int L, int C, int G, const float *gamma, const float *beta, float eps, float *y,
              float *mean, float *rstd, cudaStream_t st);
int nn_gn_bwd(const float *dy, const float *x, int N, int L, int C, int G, const float *gamma, const float *mean,
              const float *rstd, float *dx, float *dgamma_n, float *dbeta_n, cudaStream_t st);
int nn_mish(const float *x, const float *dy, float *out, long long n, int backward, cudaStream_t st);
int nn_film(const float *h, const float *film, int N, int L, int C, float *y, const float *dy, float *dh,
            float *dfilm, int backward, cudaStream_t st);
int nn_axpby(float a, const float *x, float b, const float *y, float *out, long long n, cudaStream_t st);
int nn_copy_cols(const float *in, long long R, int Cin, int in_stride, int in_off, float *out, int out_stride,
                 int out_off, int accumulate, cudaStream_t st);
int nn_upsample2(const float *x, int N, int L, int C, float *y, int backward, cudaStream_t st);
int nn_gather(const float *in, const int *idx, float *out, long long n, long long per, int scatter, cudaStream_t st);
int nn_sinusoid(const int *k, int N, int dim, float *out, cudaStream_t st);
int nn_gather_rows(const float *in, const int *rows, long long R, int C, float *out, cudaStream_t st);
int nn_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
            float wd, int step, cudaStream_t st);
int nn_ddpm_noise(const float *x0, const float *eps, const int *k, const float *abar, int N, int per, float *xk,
                  cudaStream_t st);
int nn_mse(const float *pred, const float *target, const float *w, int N, int per, float *dpred, float *loss_partial,
           int blocks, cudaStream_t st);
int nn_ddim_step(const float *xk, const float *eps, float ab_k, float ab_prev, long long n, float clip, float *out,
                 cudaStream_t st);
int nn_to_bf16(const float *x, void *y, long long n, cudaStream_t st);
int nn_clamp_affine(const float *x, float a, float b, float lo, float hi, float *out, long long n, cudaStream_t st);
int nn_conv_tc(const DseedConvTc &d, cudaStream_t st);
bool tc_maps_available();
int nn_im2col1d_bf16(const void *x, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad, void *cols,
                     cudaStream_t st);
int nn_upsample2_bf16(const void *x, int N, int L, int C, void *y, cudaStream_t st);
}  // namespace dseed

using dseed::set_error;

namespace {
int cu(int e, const char *what) {
    if (e == cudaSuccess) return DSEED_OK;
    return set_error(DSEED_ECUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)e));
}
#define NEED(cond, msg) \
    if (!(cond)) return set_error(DSEED_EINVAL, "%s", msg)
}  // namespace

extern "C" {

int dseed_nn_gemm_f32(int trans_a, int trans_b, int M, int N, int K, float alpha, const float *A_dev, int lda,
                      const float *B_dev, int ldb, float beta, float *C_dev, int ldc, const float *bias_dev,
                      cudaStream_t stream) {
    NEED(M >= 0 && N >= 0 && K >= 0, "gemm: negative size");
    NEED(N <= 65535 * 64, "gemm: N above 4194240 (column tiles in the grid's y)");
    NEED((M == 0 || N == 0) || (C_dev && (K == 0 || (A_dev && B_dev))), "gemm: NULL operand");
    return cu(dseed::nn_gemm_f32(trans_a, trans_b, M, N, K, alpha, A_dev, lda, B_dev, ldb, beta, C_dev, ldc, bias_dev,
                                 stream), "gemm_f32");
}

int dseed_nn_gemm_bf16(int M, int N, int K, const void *A_dev, const void *W_dev, float *C_dev,
                       const float *bias_dev, cudaStream_t stream) {
    NEED(M >= 0 && N >= 0 && K >= 0 && K % 16 == 0, "gemm_bf16: sizes must be >= 0 and K a multiple of 16");
    NEED(N <= 65535 * 64, "gemm_bf16: N above 4194240 (column tiles in the grid's y)");
    NEED((M == 0 || N == 0) || (A_dev && W_dev && C_dev), "gemm_bf16: NULL operand");
    return cu(dseed::nn_gemm_bf16(M, N, K, A_dev, W_dev, C_dev, bias_dev, stream), "gemm_bf16");
}

int dseed_nn_im2col1d(const float *x_dev, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad,
                      void *cols_dev, int bf16, cudaStream_t stream) {
    NEED(N >= 0 && L >= 1 && C >= 1 && k >= 1 && s >= 1 && p >= 0 && Lo >= 0 && kc_pad >= k * C, "im2col: bad shape");
    NEED(x_dev && cols_dev, "im2col: NULL pointer");
    return cu(dseed::nn_im2col1d(x_dev, N, L, C, k, s, p, Lo, kc_pad, cols_dev, bf16, stream), "im2col");
}

int dseed_nn_col2im1d(const float *cols_dev, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad,
                      float *dx_dev, cudaStream_t stream) {
    NEED(N >= 0 && L >= 1 && C >= 1 && k >= 1 && s >= 1 && p >= 0 && Lo >= 0 && kc_pad >= k * C, "col2im: bad shape");
    NEED(cols_dev && dx_dev, "col2im: NULL pointer");
    return cu(dseed::nn_col2im1d(cols_dev, N, L, C, k, s, p, Lo, kc_pad, dx_dev, stream), "col2im");
}

int dseed_nn_colsum(const float *y_dev, int R, int C, float *out_dev, int accumulate, cudaStream_t stream) {
    NEED(R >= 0 && C >= 1 && y_dev && out_dev, "colsum: bad arguments");
    NEED(C <= 65535 * 32, "colsum: C above 2097120 (column blocks in the grid's y)");
    return cu(dseed::nn_colsum(y_dev, R, C, out_dev, accumulate, stream), "colsum");
}

int dseed_nn_groupnorm_fwd(const float *x_dev, int N, int L, int C, int G, const float *gamma_dev,
                           const float *beta_dev, float eps, float *y_dev, float *mean_dev, float *rstd_dev,
                           cudaStream_t stream) {
    NEED(N >= 1 && L >= 1 && G >= 1 && C % G == 0 && C / G <= 256, "groupnorm: bad shape");
    NEED(x_dev && gamma_dev && beta_dev && y_dev && mean_dev && rstd_dev, "groupnorm: NULL pointer");
    return cu(dseed::nn_gn_fwd(x_dev, N, L, C, G, gamma_dev, beta_dev, eps, y_dev, mean_dev, rstd_dev, stream), "gn");
}

int dseed_nn_groupnorm_bwd(const float *dy_dev, const float *x_dev, int N, int L, int C, int G,
                           const float *gamma_dev, const float *mean_dev, const float *rstd_dev, float *dx_dev,
                           float *dgamma_n_dev, float *dbeta_n_dev, cudaStream_t stream) {
    NEED(N >= 1 && L >= 1 && G >= 1 && C % G == 0 && C / G <= 256, "groupnorm: bad shape");
    NEED(dy_dev && x_dev && gamma_dev && mean_dev && rstd_dev && dx_dev && dgamma_n_dev && dbeta_n_dev,
         "groupnorm: NULL pointer");
    return cu(dseed::nn_gn_bwd(dy_dev, x_dev, N, L, C, G, gamma_dev, mean_dev, rstd_dev, dx_dev, dgamma_n_dev,
                               dbeta_n_dev, stream), "gn_bwd");
}

int dseed_nn_mish(const float *x_dev, const float *dy_dev, float *out_dev, long long n, int backward,
                  cudaStream_t stream) {
    NEED(n >= 0 && x_dev && out_dev && (!backward || dy_dev), "mish: bad arguments");
    return cu(dseed::nn_mish(x_dev, dy_dev, out_dev, n, backward, stream), "mish");
}

int dseed_nn_film(const float *h_dev, const float *film_dev, int N, int L, int C, float *y_dev, const float *dy_dev,
                  float *dh_dev, float *dfilm_dev, int backward, cudaStream_t stream) {
    NEED(N >= 0 && L >= 1 && C >= 1 && h_dev && film_dev, "film: bad arguments");
    NEED(backward ? (dy_dev && dh_dev && dfilm_dev) : (y_dev != nullptr), "film: NULL output");
    return cu(dseed::nn_film(h_dev, film_dev, N, L, C, y_dev, dy_dev, dh_dev, dfilm_dev, backward, stream), "film");
}

int dseed_nn_axpby(float a, const float *x_dev, float b, const float *y_dev, float *out_dev, long long n,
                   cudaStream_t stream) {
    NEED(n >= 0 && x_dev && out_dev, "axpby: bad arguments");
    return cu(dseed::nn_axpby(a, x_dev, b, y_dev, out_dev, n, stream), "axpby");
}

int dseed_nn_copy_cols(const float *in_dev, long long R, int C_in, int in_stride, int in_off, float *out_dev,
                       int out_stride, int out_off, int accumulate, cudaStream_t stream) {
    NEED(R >= 0 && C_in >= 1 && in_dev && out_dev && in_off + C_in <= in_stride && out_off + C_in <= out_stride,
         "copy_cols: bad arguments");
    return cu(dseed::nn_copy_cols(in_dev, R, C_in, in_stride, in_off, out_dev, out_stride, out_off, accumulate, stream),
              "copy_cols");
}

int dseed_nn_upsample2(const float *x_dev, int N, int L, int C, float *y_dev, int backward, cudaStream_t stream) {
    NEED(N >= 0 && L >= 1 && C >= 1 && x_dev && y_dev, "upsample2: bad arguments");
    return cu(dseed::nn_upsample2(x_dev, N, L, C, y_dev, backward, stream), "upsample2");
}

int dseed_nn_gather(const float *in_dev, const int *idx_dev, float *out_dev, long long n, long long per, int scatter,
                    cudaStream_t stream) {
    NEED(n >= 0 && per >= 1 && in_dev && idx_dev && out_dev, "gather: bad arguments");
    return cu(dseed::nn_gather(in_dev, idx_dev, out_dev, n, per, scatter, stream), "gather");
}

int dseed_nn_gather_rows(const float *in_dev, const int *rows_dev, long long R_out, int C, float *out_dev,
                         cudaStream_t stream) {
    NEED(R_out >= 0 && C >= 1 && in_dev && rows_dev && out_dev, "gather_rows: bad arguments");
    return cu(dseed::nn_gather_rows(in_dev, rows_dev, R_out, C, out_dev, stream), "gather_rows");
}

int dseed_nn_sinusoid(const int *k_dev, int N, int dim, float *out_dev, cudaStream_t stream) {
    NEED(N >= 0 && dim >= 2 && dim % 2 == 0 && k_dev && out_dev, "sinusoid: bad arguments");
    return cu(dseed::nn_sinusoid(k_dev, N, dim, out_dev, stream), "sinusoid");
}

int dseed_nn_adam(float *p_dev, const float *g_dev, float *m_dev, float *v_dev, long long n, float lr, float beta1,
                  float beta2, float eps, float weight_decay, int step, cudaStream_t stream) {
    NEED(n >= 0 && step >= 1 && p_dev && g_dev && m_dev && v_dev, "adam: bad arguments");
    return cu(dseed::nn_adam(p_dev, g_dev, m_dev, v_dev, n, lr, beta1, beta2, eps, weight_decay, step, stream), "adam");
}

int dseed_nn_ddpm_noise(const float *x0_dev, const float *eps_dev, const int *k_dev, const float *abar_dev, int N,
                        int per, float *xk_dev, cudaStream_t stream) {
    NEED(N >= 0 && per >= 1 && x0_dev && eps_dev && k_dev && abar_dev && xk_dev, "ddpm_noise: bad arguments");
    return cu(dseed::nn_ddpm_noise(x0_dev, eps_dev, k_dev, abar_dev, N, per, xk_dev, stream), "ddpm_noise");
}

int dseed_nn_mse(const float *pred_dev, const float *target_dev, const float *w_dev, int N, int per,
                 float *dpred_dev, float *loss_partial_dev, int blocks, cudaStream_t stream) {
    NEED(N >= 1 && per >= 1 && blocks >= 1 && pred_dev && target_dev && dpred_dev && loss_partial_dev,
         "mse: bad arguments");
    return cu(dseed::nn_mse(pred_dev, target_dev, w_dev, N, per, dpred_dev, loss_partial_dev, blocks, stream), "mse");
}

int dseed_nn_ddim_step(const float *xk_dev, const float *eps_dev, float ab_k, float ab_prev, long long n, float clip,
                       float *out_dev, cudaStream_t stream) {
    NEED(n >= 0 && xk_dev && eps_dev && out_dev && ab_k > 0.f && ab_k <= 1.f && ab_prev > 0.f && ab_prev <= 1.f,
         "ddim_step: bad arguments");
    return cu(dseed::nn_ddim_step(xk_dev, eps_dev, ab_k, ab_prev, n, clip, out_dev, stream), "ddim_step");
}

int dseed_nn_to_bf16(const float *x_dev, void *y_dev, long long n, cudaStream_t stream) {
    NEED(n >= 0 && x_dev && y_dev, "to_bf16: bad arguments");
    return cu(dseed::nn_to_bf16(x_dev, y_dev, n, stream), "to_bf16");
}

int dseed_nn_clamp_affine(const float *x_dev, float a, float b, float lo, float hi, float *out_dev, long long n,
                          cudaStream_t stream) {
    NEED(n >= 0 && x_dev && out_dev, "clamp_affine: bad arguments");
    return cu(dseed::nn_clamp_affine(x_dev, a, b, lo, hi, out_dev, n, stream), "clamp_affine");
}

namespace {
bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
}  // namespace

int dseed_nn_conv_tc(const DseedConvTc *d, cudaStream_t stream) {
    NEED(d, "conv_tc: NULL descriptor");
    NEED(d->n_samples >= 0 && pow2(d->L) && d->L <= 128, "conv_tc: L must be a power of two <= 128");
    NEED(d->c0 > 0 && d->c0 % 64 == 0 && d->c1 >= 0 && d->c1 % 64 == 0, "conv_tc: channels must be multiples of 64");
    NEED(d->taps >= 1 && d->taps <= 8 && d->pad >= 0 && d->pad < d->taps, "conv_tc: bad taps / pad");
    NEED(d->cout_pad == 16 || d->cout_pad == 64 || d->cout_pad == 128 || d->cout_pad == 256,
         "conv_tc: cout_pad must be 16, 64, 128 or 256");
    NEED(d->cout >= 1 && d->cout <= d->cout_pad && d->out_ld >= d->cout, "conv_tc: bad cout / out_ld");
    NEED(d->epilogue >= 0 && d->epilogue <= 2, "conv_tc: bad epilogue");
    NEED(d->a0_dev && d->w_dev && d->out_dev && (d->c1 == 0 || d->a1_dev), "conv_tc: NULL operand");
    NEED(al16(d->a0_dev) && al16(d->a1_dev) && al16(d->w_dev) && al16(d->out_dev) && al16(d->bias_dev) &&
             al16(d->gamma_dev) && al16(d->beta_dev) && al16(d->film_dev) && al16(d->res_dev) &&
             al16(d->film_add_dev),
         "conv_tc: pointers must be 16-byte aligned");
    if (d->epilogue >= 1) NEED(d->out_ld % 8 == 0, "conv_tc: BF16 output rows must be multiples of 8");
    if (d->epilogue == 2) {
        NEED(d->cout == d->cout_pad && d->cout_pad >= 64, "conv_tc: group norm needs cout = cout_pad >= 64");
        NEED(d->bias_dev && d->gamma_dev && d->beta_dev, "conv_tc: group norm needs bias, gamma and beta");
        NEED(pow2(d->rows_per_sample) && d->rows_per_sample <= 32 &&
                 ((long long)d->n_samples * d->L) % d->rows_per_sample == 0,
             "conv_tc: rows_per_sample must be a power of two <= 32 dividing the rows");
        NEED(d->gn_eps > 0.f, "conv_tc: gn_eps must be positive");
        NEED(d->film_ld == 0 || (d->film_ld >= 2 * d->cout && d->film_ld % 4 == 0),
             "conv_tc: film_ld must be 0 or a multiple of 4 >= 2 cout");
    }
    const int r = dseed::nn_conv_tc(*d, stream);
    if (r == -1) return set_error(DSEED_ECUDA, "conv_tc: tensor map encoding failed (driver entry point missing?)");
    return cu(r, "conv_tc");
}

int dseed_nn_im2col1d_bf16(const void *x_dev, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad,
                           void *cols_dev, cudaStream_t stream) {
    NEED(N >= 0 && L >= 1 && C >= 1 && k >= 1 && s >= 1 && p >= 0 && Lo >= 0 && kc_pad >= k * C && x_dev && cols_dev,
         "im2col1d_bf16: bad arguments");
    NEED(C % 8 == 0 && kc_pad % 8 == 0 && al16(x_dev) && al16(cols_dev),
         "im2col1d_bf16: C and kc_pad must be multiples of 8, pointers 16-byte aligned");
    return cu(dseed::nn_im2col1d_bf16(x_dev, N, L, C, k, s, p, Lo, kc_pad, cols_dev, stream), "im2col1d_bf16");
}

int dseed_nn_upsample2_bf16(const void *x_dev, int N, int L, int C, void *y_dev, cudaStream_t stream) {
    NEED(N >= 0 && L >= 1 && C >= 1 && x_dev && y_dev, "upsample2_bf16: bad arguments");
    NEED(C % 8 == 0 && al16(x_dev) && al16(y_dev), "upsample2_bf16: C must be a multiple of 8, pointers 16-byte aligned");
    return cu(dseed::nn_upsample2_bf16(x_dev, N, L, C, y_dev, stream), "upsample2_bf16");
}

}  // extern "C"
