// Small MLP for the learned proposal of the heuristic modes (a project
// addition; the paper cites learned optimizers only as related work).
//
// y = w4 . relu(W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3) + b4 with
// hidden width H = 256.  Inputs, weights and stored activations are BF16.
// Products accumulate in FP32 on the tensor cores (mma.sync m16n8k16,
// bf16 x bf16 -> f32).  Master weights and Adam state are FP32.
// Quantisation points (mirrored by the CPU reference that checks the
// gradients):
//   forward:  xb = bf16(x); zl = hb(l-1) Wl_b (f32); hb(l) = bf16(relu(zl + bl));
//             y = sum_j hb3[j] * w4[j] + b4 (f32, j ascending)
//   loss:     L = sum_b (y_b - t_b)^2 / (2B); dy = (y - t) / B
//   backward: dw4 = hb3^T dy; db4 = sum dy; dz3 = dy w4^T masked by hb3 > 0;
//             dzl_b = bf16(dzl); dbl = column sums of dzl (f32);
//             dWl = hb(l-1)^T dzl_b (f32); dh(l-1) = dzl_b Wl_b^T (f32),
//             dz(l-1) = dh(l-1) masked by hb(l-1) > 0.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/mpdp.h"

namespace {

constexpr int kH = 256;

// C[M x N] (f32, row-major, ldc) = A[M x K] B[K x N], A(i, k) = A[i * ars + k * acs],
// B(k, j) = B[k * brs + j * bcs].  A warp computes a 16 x 32 tile (four
// m16n8k16 products per k-step); a block of four warps covers 64 x 32.
// Every operand load is bounds-checked (outside: zero).
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                   long ars, long acs, const __nv_bfloat16* __restrict__ B, long brs,
                                                   long bcs, float* __restrict__ C, long ldc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int row0 = blockIdx.y * 64 + warp * 16;
    const int col0 = blockIdx.x * 32;
    float acc[4][4];
#pragma unroll
    for (int t = 0; t < 4; t++)
#pragma unroll
        for (int r = 0; r < 4; r++) acc[t][r] = 0.f;
    auto lda = [&](int i, int k) -> unsigned short {
        return (i < M && k < K) ? __bfloat16_as_ushort(A[(long)i * ars + (long)k * acs]) : (unsigned short)0;
    };
    auto ldb = [&](int k, int j) -> unsigned short {
        return (k < K && j < N) ? __bfloat16_as_ushort(B[(long)k * brs + (long)j * bcs]) : (unsigned short)0;
    };
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + tq * 2;
        const uint32_t a0 = lda(row0 + g, ka) | ((uint32_t)lda(row0 + g, ka + 1) << 16);
        const uint32_t a1 = lda(row0 + g + 8, ka) | ((uint32_t)lda(row0 + g + 8, ka + 1) << 16);
        const uint32_t a2 = lda(row0 + g, ka + 8) | ((uint32_t)lda(row0 + g, ka + 9) << 16);
        const uint32_t a3 = lda(row0 + g + 8, ka + 8) | ((uint32_t)lda(row0 + g + 8, ka + 9) << 16);
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int j = col0 + t * 8 + g;
            const uint32_t b0 = ldb(ka, j) | ((uint32_t)ldb(ka + 1, j) << 16);
            const uint32_t b1 = ldb(ka + 8, j) | ((uint32_t)ldb(ka + 9, j) << 16);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[t][0]), "+f"(acc[t][1]), "+f"(acc[t][2]), "+f"(acc[t][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
    }
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int j = col0 + t * 8 + tq * 2;
        const int i0 = row0 + g, i1 = row0 + g + 8;
        if (i0 < M && j < N) C[(long)i0 * ldc + j] = acc[t][0];
        if (i0 < M && j + 1 < N) C[(long)i0 * ldc + j + 1] = acc[t][1];
        if (i1 < M && j < N) C[(long)i1 * ldc + j] = acc[t][2];
        if (i1 < M && j + 1 < N) C[(long)i1 * ldc + j + 1] = acc[t][3];
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// hb = bf16(relu(z + b)), z [M x H]
__global__ void k_bias_relu(const float* __restrict__ z, const float* __restrict__ b, __nv_bfloat16* __restrict__ hb,
                            long M)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < M * kH; i += (long)gridDim.x * blockDim.x) {
        const float v = z[i] + b[i % kH];
        hb[i] = __float2bfloat16_rn(v > 0.f ? v : 0.f);
    }
}

// y[b] = sum_j hb3[b, j] * w4[j] + b4 (j ascending, one thread per row)
__global__ void k_head(const __nv_bfloat16* __restrict__ hb, const float* __restrict__ w4, const float* __restrict__ b4,
                       float* __restrict__ y, int M)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= M) return;
    float s = 0.f;
    for (int j = 0; j < kH; j++) s = __fadd_rn(s, __fmul_rn(__bfloat162float(hb[(long)b * kH + j]), w4[j]));
    y[b] = __fadd_rn(s, b4[0]);
}

// dy = (y - t) / M; dz3 = dy w4^T masked by hb3 > 0 (f32 and bf16); also the
// per-row loss terms
__global__ void k_head_back(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ w4,
                            const __nv_bfloat16* __restrict__ hb3, float* __restrict__ dy, float* __restrict__ dz,
                            __nv_bfloat16* __restrict__ dzb, float* __restrict__ lossterm, int M)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)M * kH; i += (long)gridDim.x * blockDim.x) {
        const int b = (int)(i / kH), j = (int)(i % kH);
        const float d = __fsub_rn(y[b], t[b]);
        const float g = __fdiv_rn(d, (float)M);
        if (j == 0) {
            dy[b] = g;
            lossterm[b] = __fmul_rn(d, d);
        }
        const float v = __bfloat162float(hb3[i]) > 0.f ? __fmul_rn(g, w4[j]) : 0.f;
        dz[i] = v;
        dzb[i] = __float2bfloat16_rn(v);
    }
}

// dz = dh masked by hb > 0 (f32 and bf16)
__global__ void k_relu_back(const float* __restrict__ dh, const __nv_bfloat16* __restrict__ hb, float* __restrict__ dz,
                            __nv_bfloat16* __restrict__ dzb, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float v = __bfloat162float(hb[i]) > 0.f ? dh[i] : 0.f;
        dz[i] = v;
        dzb[i] = __float2bfloat16_rn(v);
    }
}

// out[j] = sum_b x[b, j] (rows ascending), one thread per column
__global__ void k_colsum(const float* __restrict__ x, float* __restrict__ out, int M, int N)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    float s = 0.f;
    for (int b = 0; b < M; b++) s = __fadd_rn(s, x[(long)b * N + j]);
    out[j] = s;
}

// dw4[j] = sum_b dy[b] * hb3[b, j]
__global__ void k_head_wgrad(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ hb3, float* __restrict__ dw4,
                             int M)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kH) return;
    float s = 0.f;
    for (int b = 0; b < M; b++) s = __fadd_rn(s, __fmul_rn(dy[b], __bfloat162float(hb3[(long)b * kH + j])));
    dw4[j] = s;
}

// Adam on the f32 master parameters, then their bf16 copies
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        m[i] = b1 * m[i] + (1.f - b1) * gi;
        v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
        const float mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

}  // namespace

// Parameter layout (f32, contiguous): W1 [F x H], b1 [H], W2 [H x H], b2 [H],
// W3 [H x H], b3 [H], w4 [H], b4 [1]; F = the input width.
struct mpdp_mlp {
    int device = 0;
    int F = 0;
    long P = 0;
    long off[8] = {};
    float* params = nullptr;  // device, f32 masters
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* wb = nullptr;  // bf16 copies of W1, W2, W3 (same offsets as in params for these three)
    long steps = 0;
    // activations for a batch of up to cap rows
    int cap = 0;
    void* act = nullptr;
    cudaStream_t stream = nullptr;
};

namespace {

int ensure_act(mpdp_mlp* m, int M)
{
    if (M <= m->cap) return MPDP_OK;
    if (m->act) cudaFree(m->act);
    m->act = nullptr;
    m->cap = 0;
    const size_t rows = (size_t)M;
    // xb, hb1, hb2, hb3 (bf16) + z (f32 H) + dz (f32 H) + dzb (bf16 H) + dh (f32 H) + y, dy, loss (f32)
    const size_t bytes = rows * (size_t)m->F * 2 + 3 * rows * kH * 2 + rows * kH * 4 * 3 + rows * kH * 2 +
                         rows * 4 * 3 + 16 * 256;
    if (cudaMalloc(&m->act, bytes) != cudaSuccess) {
        cudaGetLastError();
        m->act = nullptr;
        return MPDP_ERR_OOM;
    }
    m->cap = M;
    return MPDP_OK;
}

struct Act {
    __nv_bfloat16 *xb, *hb1, *hb2, *hb3, *dzb;
    float *z, *dz, *dh, *y, *dy, *loss;
};

Act act_of(mpdp_mlp* m)
{
    char* c = static_cast<char*>(m->act);
    const size_t rows = (size_t)m->cap;
    Act a;
    auto take = [&](size_t bytes) {
        char* r = c;
        c += (bytes + 255) & ~(size_t)255;
        return r;
    };
    a.xb = reinterpret_cast<__nv_bfloat16*>(take(rows * m->F * 2));
    a.hb1 = reinterpret_cast<__nv_bfloat16*>(take(rows * kH * 2));
    a.hb2 = reinterpret_cast<__nv_bfloat16*>(take(rows * kH * 2));
    a.hb3 = reinterpret_cast<__nv_bfloat16*>(take(rows * kH * 2));
    a.dzb = reinterpret_cast<__nv_bfloat16*>(take(rows * kH * 2));
    a.z = reinterpret_cast<float*>(take(rows * kH * 4));
    a.dz = reinterpret_cast<float*>(take(rows * kH * 4));
    a.dh = reinterpret_cast<float*>(take(rows * kH * 4));
    a.y = reinterpret_cast<float*>(take(rows * 4));
    a.dy = reinterpret_cast<float*>(take(rows * 4));
    a.loss = reinterpret_cast<float*>(take(rows * 4));
    return a;
}

void gemm(cudaStream_t st, int M, int N, int K, const __nv_bfloat16* A, long ars, long acs, const __nv_bfloat16* B,
          long brs, long bcs, float* C, long ldc)
{
    dim3 grid((N + 31) / 32, (M + 63) / 64);
    k_gemm_bf16<<<grid, 128, 0, st>>>(M, N, K, A, ars, acs, B, brs, bcs, C, ldc);
}

int grid_for(long n) { return (int)std::min<long>((n + 255) / 256, 4096); }

void refresh_bf16(mpdp_mlp* m)
{
    for (int l = 0; l < 3; l++) {
        const long o = m->off[2 * l], n = m->off[2 * l + 1] - o;
        k_to_bf16<<<grid_for(n), 256, 0, m->stream>>>(m->params + o, m->wb + o, n);
    }
}

// forward for rows [0, M): leaves hb1..hb3 and y in the activation buffers
void forward(mpdp_mlp* m, const float* x, int M, const Act& a)
{
    cudaStream_t st = m->stream;
    const float* P = m->params;
    k_to_bf16<<<grid_for((long)M * m->F), 256, 0, st>>>(x, a.xb, (long)M * m->F);
    gemm(st, M, kH, m->F, a.xb, m->F, 1, m->wb + m->off[0], kH, 1, a.z, kH);
    k_bias_relu<<<grid_for((long)M * kH), 256, 0, st>>>(a.z, P + m->off[1], a.hb1, M);
    gemm(st, M, kH, kH, a.hb1, kH, 1, m->wb + m->off[2], kH, 1, a.z, kH);
    k_bias_relu<<<grid_for((long)M * kH), 256, 0, st>>>(a.z, P + m->off[3], a.hb2, M);
    gemm(st, M, kH, kH, a.hb2, kH, 1, m->wb + m->off[4], kH, 1, a.z, kH);
    k_bias_relu<<<grid_for((long)M * kH), 256, 0, st>>>(a.z, P + m->off[5], a.hb3, M);
    k_head<<<(M + 127) / 128, 128, 0, st>>>(a.hb3, P + m->off[6], P + m->off[7], a.y, M);
}

// gradients of the batch into m->grads (and the summed squared errors)
void backward(mpdp_mlp* m, const float* t, int M, const Act& a)
{
    cudaStream_t st = m->stream;
    float* G = m->grads;
    const float* P = m->params;
    k_head_back<<<grid_for((long)M * kH), 256, 0, st>>>(a.y, t, P + m->off[6], a.hb3, a.dy, a.dz, a.dzb, a.loss, M);
    k_head_wgrad<<<1, kH, 0, st>>>(a.dy, a.hb3, G + m->off[6], M);
    k_colsum<<<1, 32, 0, st>>>(a.dy, G + m->off[7], M, 1);
    const __nv_bfloat16* hprev[3] = {a.xb, a.hb1, a.hb2};
    for (int l = 2; l >= 0; l--) {
        const int K = l == 0 ? m->F : kH;  // rows of Wl
        // dbl = column sums of dzl; dWl = hprev^T dzl_b
        k_colsum<<<1, kH, 0, st>>>(a.dz, G + m->off[2 * l + 1], M, kH);
        gemm(st, K, kH, M, hprev[l], 1, K, a.dzb, kH, 1, G + m->off[2 * l], kH);
        if (l == 0) break;
        // dh(l-1) = dzl_b Wl_b^T, then dz(l-1) masked by hb(l-1) > 0
        gemm(st, M, kH, kH, a.dzb, kH, 1, m->wb + m->off[2 * l], 1, kH, a.dh, kH);
        k_relu_back<<<grid_for((long)M * kH), 256, 0, st>>>(a.dh, hprev[l], a.dz, a.dzb, (long)M * kH);
    }
}

}  // namespace

extern "C" {

int mpdp_mlp_create(mpdp_mlp** out, int device, int32_t n_in, void* cuda_stream)
{
    if (!out || n_in < 1 || n_in > 1024) return MPDP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    mpdp_mlp* m = new mpdp_mlp();
    m->device = device;
    m->F = n_in;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    const long sizes[8] = {(long)n_in * kH, kH, (long)kH * kH, kH, (long)kH * kH, kH, kH, 1};
    long o = 0;
    for (int i = 0; i < 8; i++) {
        m->off[i] = o;
        o += sizes[i];
    }
    m->P = o;
    const size_t bytes = (size_t)o * 4;
    if (cudaMalloc(&m->params, bytes) != cudaSuccess || cudaMalloc(&m->grads, bytes) != cudaSuccess ||
        cudaMalloc(&m->adam_m, bytes) != cudaSuccess || cudaMalloc(&m->adam_v, bytes) != cudaSuccess ||
        cudaMalloc(&m->wb, (size_t)o * 2) != cudaSuccess) {
        cudaGetLastError();
        mpdp_mlp_destroy(m);
        return MPDP_ERR_OOM;
    }
    cudaMemsetAsync(m->params, 0, bytes, m->stream);
    cudaMemsetAsync(m->grads, 0, bytes, m->stream);
    cudaMemsetAsync(m->adam_m, 0, bytes, m->stream);
    cudaMemsetAsync(m->adam_v, 0, bytes, m->stream);
    cudaMemsetAsync(m->wb, 0, (size_t)o * 2, m->stream);
    if (cudaGetLastError() != cudaSuccess) {
        mpdp_mlp_destroy(m);
        return MPDP_ERR_CUDA;
    }
    *out = m;
    return MPDP_OK;
}

void mpdp_mlp_destroy(mpdp_mlp* m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    cudaFree(m->params);
    cudaFree(m->grads);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->wb);
    if (m->act) cudaFree(m->act);
    cudaGetLastError();
    delete m;
}

int64_t mpdp_mlp_param_count(const mpdp_mlp* m) { return m ? m->P : 0; }

int mpdp_mlp_set_params(mpdp_mlp* m, const float* host, int64_t count)
{
    if (!m || !host || count != m->P) return MPDP_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    if (cudaMemcpyAsync(m->params, host, (size_t)count * 4, cudaMemcpyHostToDevice, m->stream) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    refresh_bf16(m);
    m->steps = 0;
    cudaMemsetAsync(m->adam_m, 0, (size_t)count * 4, m->stream);
    cudaMemsetAsync(m->adam_v, 0, (size_t)count * 4, m->stream);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? MPDP_OK : MPDP_ERR_CUDA;
}

int mpdp_mlp_get_params(mpdp_mlp* m, float* host, int64_t count)
{
    if (!m || !host || count != m->P) return MPDP_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    if (cudaMemcpyAsync(host, m->params, (size_t)count * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess) {
        cudaGetLastError();
        return MPDP_ERR_CUDA;
    }
    return MPDP_OK;
}

int mpdp_mlp_forward(mpdp_mlp* m, const float* d_x, int32_t rows, float* d_y)
{
    if (!m || rows < 0 || (rows > 0 && (!d_x || !d_y))) return MPDP_ERR_INVALID_ARG;
    if (rows == 0) return MPDP_OK;
    cudaSetDevice(m->device);
    const int rc = ensure_act(m, rows);
    if (rc != MPDP_OK) return rc;
    const Act a = act_of(m);
    forward(m, d_x, rows, a);
    if (cudaMemcpyAsync(d_y, a.y, (size_t)rows * 4, cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
        return MPDP_ERR_CUDA;
    return MPDP_OK;
}

int mpdp_mlp_gradients(mpdp_mlp* m, const float* d_x, const float* d_t, int32_t rows, float* host_grads,
                       double* loss)
{
    if (!m || rows < 1 || !d_x || !d_t) return MPDP_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    const int rc = ensure_act(m, rows);
    if (rc != MPDP_OK) return rc;
    const Act a = act_of(m);
    forward(m, d_x, rows, a);
    backward(m, d_t, rows, a);
    if (host_grads &&
        cudaMemcpyAsync(host_grads, m->grads, (size_t)m->P * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return MPDP_ERR_CUDA;
    if (loss) {
        std::vector<float> lt(rows);
        if (cudaMemcpyAsync(lt.data(), a.loss, (size_t)rows * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
            return MPDP_ERR_CUDA;
        if (cudaStreamSynchronize(m->stream) != cudaSuccess) return MPDP_ERR_CUDA;
        double s = 0.0;
        for (int i = 0; i < rows; i++) s += lt[i];
        *loss = s / (2.0 * rows);
    }
    if (cudaStreamSynchronize(m->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) return MPDP_ERR_CUDA;
    return MPDP_OK;
}

int mpdp_mlp_train_step(mpdp_mlp* m, const float* d_x, const float* d_t, int32_t rows, float lr)
{
    if (!m || rows < 1 || !d_x || !d_t || !(lr > 0.f)) return MPDP_ERR_INVALID_ARG;
    cudaSetDevice(m->device);
    const int rc = ensure_act(m, rows);
    if (rc != MPDP_OK) return rc;
    const Act a = act_of(m);
    forward(m, d_x, rows, a);
    backward(m, d_t, rows, a);
    m->steps++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->steps), c2 = 1.f - powf(b2, (float)m->steps);
    k_adam<<<grid_for(m->P), 256, 0, m->stream>>>(m->params, m->grads, m->adam_m, m->adam_v, m->P, lr, b1, b2, 1e-8f,
                                                   c1, c2);
    refresh_bf16(m);
    return cudaGetLastError() == cudaSuccess ? MPDP_OK : MPDP_ERR_CUDA;
}

}  // extern "C"
