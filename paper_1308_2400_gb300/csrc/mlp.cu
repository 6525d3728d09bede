// Small MLP cost model for the batch dispatcher: forward, MSE loss,
// backward and Adam on the GPU.  The network maps F instance features to
// V predicted log-times (one per kernel variant):
//   H1 = relu(X W1 + b1),  H2 = relu(H1 W2 + b2),  P = H2 W3 + b3,
// parameters stored flat as [W1 (F x H), b1 (H), W2 (H x H), b2 (H),
// W3 (H x V), b3 (V)], row-major.  The loss is the mean over observed
// targets of (P - T)^2 (mask M = 1 where T was measured).
// Sizes are tiny (F ~ 10, H <= 64, rows ~ 1e3-1e4): one thread per output
// element, FP32.
#include "afmm_common.cuh"

namespace afmm {
namespace {

constexpr int kT = 256;

inline unsigned blocks(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

// out[r, o] = act(sum_i in[r, i] W[i, o] + b[o])
__global__ void dense_fwd(const float* __restrict__ in, const float* __restrict__ W,
                          const float* __restrict__ b, float* __restrict__ out,
                          int rows, int din, int dout, int relu) {
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)rows * dout) return;
    const int r = (int)(t / dout), o = (int)(t % dout);
    float s = b[o];
    for (int i = 0; i < din; ++i) s = fmaf(in[(int64_t)r * din + i], W[(int64_t)i * dout + o], s);
    out[t] = relu ? fmaxf(s, 0.f) : s;
}

// dP = 2 M (P - T) / count;  loss partials
__global__ void mse_grad(const float* __restrict__ P, const float* __restrict__ T,
                         const float* __restrict__ M, float* __restrict__ dP,
                         int64_t n, float inv_count, float* __restrict__ loss) {
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    float l = 0.f;
    if (t < n) {
        const float d = (P[t] - T[t]) * M[t];
        dP[t] = 2.f * d * inv_count;
        l = d * d * inv_count;
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// dW[i, o] = sum_r in[r, i] dout[r, o];  db[o] = sum_r dout[r, o]
__global__ void dense_bwd_w(const float* __restrict__ in, const float* __restrict__ dO,
                            float* __restrict__ dW, float* __restrict__ db, int rows,
                            int din, int dout) {
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    const int64_t nw = (int64_t)din * dout;
    if (t < nw) {
        const int i = (int)(t / dout), o = (int)(t % dout);
        float s = 0.f;
        for (int r = 0; r < rows; ++r) s = fmaf(in[(int64_t)r * din + i], dO[(int64_t)r * dout + o], s);
        dW[t] = s;
    } else if (t < nw + dout) {
        const int o = (int)(t - nw);
        float s = 0.f;
        for (int r = 0; r < rows; ++r) s += dO[(int64_t)r * dout + o];
        db[o] = s;
    }
}

// din[r, i] = (sum_o dout[r, o] W[i, o]) * (act[r, i] > 0)
__global__ void dense_bwd_x(const float* __restrict__ dO, const float* __restrict__ W,
                            const float* __restrict__ act, float* __restrict__ dI, int rows,
                            int din, int dout) {
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= (int64_t)rows * din) return;
    const int r = (int)(t / din), i = (int)(t % din);
    float s = 0.f;
    for (int o = 0; o < dout; ++o) s = fmaf(dO[(int64_t)r * dout + o], W[(int64_t)i * dout + o], s);
    dI[t] = act[t] > 0.f ? s : 0.f;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
    const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
    if (t >= n) return;
    const float gt = g[t];
    const float mt = b1 * m[t] + (1.f - b1) * gt;
    const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
    m[t] = mt;
    v[t] = vt;
    p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
}

struct Offs {
    int64_t W1, b1, W2, b2, W3, b3, total;
};
Offs offsets(const afmm_mlp_shape& s) {
    Offs o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)s.features * s.hidden;
    o.W2 = o.b1 + s.hidden;
    o.b2 = o.W2 + (int64_t)s.hidden * s.hidden;
    o.W3 = o.b2 + s.hidden;
    o.b3 = o.W3 + (int64_t)s.hidden * s.outputs;
    o.total = o.b3 + s.outputs;
    return o;
}

bool shape_ok(const afmm_mlp_shape* s) {
    return s && s->features > 0 && s->hidden > 0 && s->outputs > 0 &&
           s->features <= 1024 && s->hidden <= 1024 && s->outputs <= 64;
}

}  // namespace

int64_t mlp_param_count(const afmm_mlp_shape& s) { return offsets(s).total; }
int64_t mlp_work_floats(const afmm_mlp_shape& s, int rows) {
    // H1, H2, P, dP, dH2, dH1
    return (int64_t)rows * (3 * s.hidden + 2 * s.outputs + s.hidden);
}

afmm_status mlp_forward(const afmm_mlp_shape& s, const float* params, const float* X,
                        int rows, float* P, float* work, cudaStream_t st) {
    const Offs o = offsets(s);
    float* H1 = work;
    float* H2 = H1 + (int64_t)rows * s.hidden;
    dense_fwd<<<blocks((int64_t)rows * s.hidden), kT, 0, st>>>(X, params + o.W1, params + o.b1,
                                                              H1, rows, s.features, s.hidden, 1);
    dense_fwd<<<blocks((int64_t)rows * s.hidden), kT, 0, st>>>(H1, params + o.W2, params + o.b2,
                                                              H2, rows, s.hidden, s.hidden, 1);
    dense_fwd<<<blocks((int64_t)rows * s.outputs), kT, 0, st>>>(H2, params + o.W3, params + o.b3,
                                                               P, rows, s.hidden, s.outputs, 0);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(3);
    return AFMM_OK;
}

afmm_status mlp_loss_grad(const afmm_mlp_shape& s, const float* params, const float* X,
                          const float* T, const float* M, int rows, float count,
                          float* grads, float* work, float* loss, cudaStream_t st) {
    const Offs o = offsets(s);
    float* H1 = work;
    float* H2 = H1 + (int64_t)rows * s.hidden;
    float* P = H2 + (int64_t)rows * s.hidden;
    float* dP = P + (int64_t)rows * s.outputs;
    float* dH2 = dP + (int64_t)rows * s.outputs;
    float* dH1 = dH2 + (int64_t)rows * s.hidden;
    AFMM_TRY(mlp_forward(s, params, X, rows, P, work, st));
    AFMM_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    const int64_t np = (int64_t)rows * s.outputs;
    mse_grad<<<blocks(np), kT, 0, st>>>(P, T, M, dP, np, count > 0 ? 1.f / count : 0.f, loss);
    dense_bwd_w<<<blocks((int64_t)s.hidden * s.outputs + s.outputs), kT, 0, st>>>(
        H2, dP, grads + o.W3, grads + o.b3, rows, s.hidden, s.outputs);
    dense_bwd_x<<<blocks((int64_t)rows * s.hidden), kT, 0, st>>>(dP, params + o.W3, H2, dH2,
                                                                rows, s.hidden, s.outputs);
    dense_bwd_w<<<blocks((int64_t)s.hidden * s.hidden + s.hidden), kT, 0, st>>>(
        H1, dH2, grads + o.W2, grads + o.b2, rows, s.hidden, s.hidden);
    dense_bwd_x<<<blocks((int64_t)rows * s.hidden), kT, 0, st>>>(dH2, params + o.W2, H1, dH1,
                                                                rows, s.hidden, s.hidden);
    dense_bwd_w<<<blocks((int64_t)s.features * s.hidden + s.hidden), kT, 0, st>>>(
        X, dH1, grads + o.W1, grads + o.b1, rows, s.features, s.hidden);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(6);
    return AFMM_OK;
}

afmm_status mlp_adam(int64_t n, float* params, const float* grads, float* m, float* v,
                     float lr, float b1, float b2, float eps, int step, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<blocks(n), kT, 0, st>>>(params, grads, m, v, n, lr, b1, b2, eps, c1, c2);
    AFMM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return AFMM_OK;
}

}  // namespace afmm
