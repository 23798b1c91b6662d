// k_mlp.cu -- the learned planner's network on the GPU: forward pass,
// backward pass and Adam update, written as plain CUDA kernels (fp32).
//
// Network: x -> h1 = relu(W1 x + b1) -> h2 = relu(W2 h1 + b2) -> y = W3 h2 + b3.
// Loss on a batch: L = sum(mask (y - t)^2) / sum(mask).
// Backward: dy = 2 mask (y - t) / sum(mask); for a layer y = act(W x + b):
//   dz = dy * act'(z),  dW = dz^T x,  db = sum_rows dz,  dx = dz W.
// Each output element of every kernel is produced by one thread summing in a
// fixed order, so training is deterministic for a given seed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "gett_learn.h"
#include "internal.h"

struct gett_mlp {
    int nfeat = 0, hidden = 0, nout = 0;
    int np = 0;
    float *p = nullptr;   // parameters
    float *g = nullptr;   // gradients
    float *m1 = nullptr;  // Adam first moment
    float *m2 = nullptr;  // Adam second moment
    int step = 0;
    // activations for a batch of up to cap rows
    int cap = 0;
    float *x = nullptr, *h1 = nullptr, *h2 = nullptr, *y = nullptr, *t = nullptr, *mask = nullptr;
    float *dy = nullptr, *dh2 = nullptr, *dh1 = nullptr;
    float *loss = nullptr;
};

namespace {

using gett::set_last_cuda_error;

struct Offs {
    size_t W1, b1, W2, b2, W3, b3, total;
};

Offs offsets(int nf, int h, int no)
{
    Offs o;
    o.W1 = 0;
    o.b1 = o.W1 + (size_t)h * nf;
    o.W2 = o.b1 + h;
    o.b2 = o.W2 + (size_t)h * h;
    o.W3 = o.b2 + h;
    o.b3 = o.W3 + (size_t)no * h;
    o.total = o.b3 + no;
    return o;
}

// Y[r][o] = act(sum_i X[r][i] W[o][i] + b[o])
__global__ void linear_fwd(const float *__restrict__ X, const float *__restrict__ W, const float *__restrict__ b,
                           float *__restrict__ Y, int rows, int in, int out, int relu)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * out) return;
    const int r = idx / out, o = idx % out;
    float s = b[o];
    const float *x = X + (size_t)r * in;
    const float *w = W + (size_t)o * in;
    for (int i = 0; i < in; ++i) s = fmaf(x[i], w[i], s);
    Y[idx] = relu ? fmaxf(s, 0.f) : s;
}

// dy = 2 mask (y - t) / count; loss = sum mask (y - t)^2 / count (one block)
__global__ void mse_grad(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ mask,
                         float *__restrict__ dy, float *__restrict__ loss, int n)
{
    __shared__ float s_cnt[256], s_sum[256];
    float cnt = 0.f, sum = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        cnt += mask[i];
        const float d = y[i] - t[i];
        sum += mask[i] * d * d;
    }
    s_cnt[threadIdx.x] = cnt;
    s_sum[threadIdx.x] = sum;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            s_cnt[threadIdx.x] += s_cnt[threadIdx.x + st];
            s_sum[threadIdx.x] += s_sum[threadIdx.x + st];
        }
        __syncthreads();
    }
    const float c = fmaxf(s_cnt[0], 1.f);
    for (int i = threadIdx.x; i < n; i += blockDim.x) dy[i] = 2.f * mask[i] * (y[i] - t[i]) / c;
    if (threadIdx.x == 0) *loss = s_sum[0] / c;
}

// dW[o][i] = sum_r dZ[r][o] X[r][i];  db[o] = sum_r dZ[r][o]
__global__ void linear_bwd_w(const float *__restrict__ dZ, const float *__restrict__ X, float *__restrict__ dW,
                             float *__restrict__ db, int rows, int in, int out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < out * in) {
        const int o = idx / in, i = idx % in;
        float s = 0.f;
        for (int r = 0; r < rows; ++r) s = fmaf(dZ[(size_t)r * out + o], X[(size_t)r * in + i], s);
        dW[idx] = s;
    }
    if (idx < out) {
        float s = 0.f;
        for (int r = 0; r < rows; ++r) s += dZ[(size_t)r * out + idx];
        db[idx] = s;
    }
}

// dX[r][i] = (sum_o dZ[r][o] W[o][i]) * [Xact[r][i] > 0]   (ReLU of the layer below)
__global__ void linear_bwd_x(const float *__restrict__ dZ, const float *__restrict__ W,
                             const float *__restrict__ Xact, float *__restrict__ dX, int rows, int in, int out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * in) return;
    const int r = idx / in, i = idx % in;
    float s = 0.f;
    for (int o = 0; o < out; ++o) s = fmaf(dZ[(size_t)r * out + o], W[(size_t)o * in + i], s);
    dX[idx] = Xact[idx] > 0.f ? s : 0.f;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int blocks(int n) { return (n + 255) / 256; }

cudaError_t ensure_cap(gett_mlp *m, int rows)
{
    if (rows <= m->cap) return cudaSuccess;
    float **bufs[] = {&m->x, &m->h1, &m->h2, &m->y, &m->t, &m->mask, &m->dy, &m->dh2, &m->dh1};
    for (float **b : bufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    const size_t R = (size_t)rows;
    cudaError_t e = cudaMalloc(&m->x, 4 * R * m->nfeat);
    if (e == cudaSuccess) e = cudaMalloc(&m->h1, 4 * R * m->hidden);
    if (e == cudaSuccess) e = cudaMalloc(&m->h2, 4 * R * m->hidden);
    if (e == cudaSuccess) e = cudaMalloc(&m->y, 4 * R * m->nout);
    if (e == cudaSuccess) e = cudaMalloc(&m->t, 4 * R * m->nout);
    if (e == cudaSuccess) e = cudaMalloc(&m->mask, 4 * R * m->nout);
    if (e == cudaSuccess) e = cudaMalloc(&m->dy, 4 * R * m->nout);
    if (e == cudaSuccess) e = cudaMalloc(&m->dh2, 4 * R * m->hidden);
    if (e == cudaSuccess) e = cudaMalloc(&m->dh1, 4 * R * m->hidden);
    if (e == cudaSuccess) m->cap = rows;
    return e;
}

void forward(gett_mlp *m, int rows)
{
    const Offs o = offsets(m->nfeat, m->hidden, m->nout);
    linear_fwd<<<blocks(rows * m->hidden), 256>>>(m->x, m->p + o.W1, m->p + o.b1, m->h1, rows, m->nfeat, m->hidden, 1);
    linear_fwd<<<blocks(rows * m->hidden), 256>>>(m->h1, m->p + o.W2, m->p + o.b2, m->h2, rows, m->hidden, m->hidden, 1);
    linear_fwd<<<blocks(rows * m->nout), 256>>>(m->h2, m->p + o.W3, m->p + o.b3, m->y, rows, m->hidden, m->nout, 0);
}

void backward(gett_mlp *m, int rows)
{
    const Offs o = offsets(m->nfeat, m->hidden, m->nout);
    mse_grad<<<1, 256>>>(m->y, m->t, m->mask, m->dy, m->loss, rows * m->nout);
    // layer 3 (no activation)
    linear_bwd_w<<<blocks(m->nout * m->hidden), 256>>>(m->dy, m->h2, m->g + o.W3, m->g + o.b3, rows, m->hidden, m->nout);
    linear_bwd_x<<<blocks(rows * m->hidden), 256>>>(m->dy, m->p + o.W3, m->h2, m->dh2, rows, m->hidden, m->nout);
    // layer 2
    linear_bwd_w<<<blocks(m->hidden * m->hidden), 256>>>(m->dh2, m->h1, m->g + o.W2, m->g + o.b2, rows, m->hidden, m->hidden);
    linear_bwd_x<<<blocks(rows * m->hidden), 256>>>(m->dh2, m->p + o.W2, m->h1, m->dh1, rows, m->hidden, m->hidden);
    // layer 1
    linear_bwd_w<<<blocks(m->hidden * m->nfeat), 256>>>(m->dh1, m->x, m->g + o.W1, m->g + o.b1, rows, m->nfeat, m->hidden);
}

int fail(cudaError_t e)
{
    set_last_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? GETT_ERR_NOMEM : GETT_ERR_CUDA;
}

}  // namespace

extern "C" int gett_mlp_create(int nfeat, int hidden, int nout, unsigned long long seed, gett_mlp **out)
{
    if (!out || nfeat <= 0 || hidden <= 0 || nout <= 0) return GETT_ERR_ARG;
    gett_mlp *m = new gett_mlp();
    m->nfeat = nfeat;
    m->hidden = hidden;
    m->nout = nout;
    const Offs o = offsets(nfeat, hidden, nout);
    m->np = (int)o.total;
    cudaError_t e = cudaMalloc(&m->p, 4 * o.total);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, 4 * o.total);
    if (e == cudaSuccess) e = cudaMalloc(&m->m1, 4 * o.total);
    if (e == cudaSuccess) e = cudaMalloc(&m->m2, 4 * o.total);
    if (e == cudaSuccess) e = cudaMalloc(&m->loss, 4);
    if (e == cudaSuccess) e = cudaMemset(m->m1, 0, 4 * o.total);
    if (e == cudaSuccess) e = cudaMemset(m->m2, 0, 4 * o.total);
    if (e != cudaSuccess) {
        gett_mlp_destroy(m);
        return fail(e);
    }
    // He-uniform initialisation from a seeded generator, biases zero
    std::vector<float> host(o.total, 0.f);
    std::mt19937_64 rng(seed);
    auto init = [&](size_t off, int fan_in, size_t count) {
        const float lim = std::sqrt(6.f / (float)fan_in);
        std::uniform_real_distribution<float> d(-lim, lim);
        for (size_t i = 0; i < count; ++i) host[off + i] = d(rng);
    };
    init(o.W1, nfeat, (size_t)hidden * nfeat);
    init(o.W2, hidden, (size_t)hidden * hidden);
    init(o.W3, hidden, (size_t)nout * hidden);
    e = cudaMemcpy(m->p, host.data(), 4 * o.total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        gett_mlp_destroy(m);
        return fail(e);
    }
    *out = m;
    return GETT_OK;
}

extern "C" int gett_mlp_destroy(gett_mlp *m)
{
    if (!m) return GETT_OK;
    float *bufs[] = {m->p, m->g, m->m1, m->m2, m->x, m->h1, m->h2, m->y, m->t, m->mask, m->dy, m->dh2, m->dh1, m->loss};
    for (float *b : bufs)
        if (b) cudaFree(b);
    delete m;
    return GETT_OK;
}

extern "C" int gett_mlp_num_params(const gett_mlp *m) { return m ? m->np : 0; }

extern "C" int gett_mlp_get_params(const gett_mlp *m, float *host)
{
    if (!m || !host) return GETT_ERR_ARG;
    cudaError_t e = cudaMemcpy(host, m->p, 4 * (size_t)m->np, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GETT_OK : fail(e);
}

extern "C" int gett_mlp_set_params(gett_mlp *m, const float *host)
{
    if (!m || !host) return GETT_ERR_ARG;
    cudaError_t e = cudaMemcpy(m->p, host, 4 * (size_t)m->np, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? GETT_OK : fail(e);
}

static cudaError_t upload_batch(gett_mlp *m, const float *X, const float *Y, const float *mask, int rows)
{
    cudaError_t e = ensure_cap(m, rows);
    if (e == cudaSuccess) e = cudaMemcpy(m->x, X, 4 * (size_t)rows * m->nfeat, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && Y) e = cudaMemcpy(m->t, Y, 4 * (size_t)rows * m->nout, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && mask) e = cudaMemcpy(m->mask, mask, 4 * (size_t)rows * m->nout, cudaMemcpyHostToDevice);
    return e;
}

extern "C" int gett_mlp_loss_grad(gett_mlp *m, const float *X, const float *Y, const float *mask, int n, float *loss,
                                  float *grads)
{
    if (!m || !X || !Y || !mask || n <= 0) return GETT_ERR_ARG;
    cudaError_t e = upload_batch(m, X, Y, mask, n);
    if (e != cudaSuccess) return fail(e);
    forward(m, n);
    backward(m, n);
    e = cudaGetLastError();
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, m->loss, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && grads) e = cudaMemcpy(grads, m->g, 4 * (size_t)m->np, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GETT_OK : fail(e);
}

extern "C" int gett_mlp_fit(gett_mlp *m, const float *X, const float *Y, const float *mask, int n, int epochs,
                            int batch, float lr, unsigned long long seed, float *final_loss)
{
    if (!m || !X || !Y || !mask || n <= 0 || epochs <= 0 || batch <= 0) return GETT_ERR_ARG;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::mt19937_64 rng(seed);
    std::vector<float> bx((size_t)batch * m->nfeat), by((size_t)batch * m->nout), bm((size_t)batch * m->nout);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        double sum = 0;
        int nb = 0;
        for (int s = 0; s < n; s += batch) {
            const int rows = std::min(batch, n - s);
            for (int r = 0; r < rows; ++r) {
                const int i = order[s + r];
                std::memcpy(&bx[(size_t)r * m->nfeat], X + (size_t)i * m->nfeat, 4 * m->nfeat);
                std::memcpy(&by[(size_t)r * m->nout], Y + (size_t)i * m->nout, 4 * m->nout);
                std::memcpy(&bm[(size_t)r * m->nout], mask + (size_t)i * m->nout, 4 * m->nout);
            }
            cudaError_t e = upload_batch(m, bx.data(), by.data(), bm.data(), rows);
            if (e != cudaSuccess) return fail(e);
            forward(m, rows);
            backward(m, rows);
            m->step++;
            const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
            adam_kernel<<<blocks(m->np), 256>>>(m->p, m->g, m->m1, m->m2, m->np, lr, b1, b2, eps, c1, c2);
            float l = 0;
            e = cudaMemcpy(&l, m->loss, 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return fail(e);
            sum += l;
            ++nb;
        }
        last = sum / std::max(nb, 1);
    }
    if (final_loss) *final_loss = (float)last;
    cudaError_t e = cudaDeviceSynchronize();
    return e == cudaSuccess ? GETT_OK : fail(e);
}

extern "C" int gett_mlp_predict(gett_mlp *m, const float *X, int n, float *Y)
{
    if (!m || !X || !Y || n <= 0) return GETT_ERR_ARG;
    cudaError_t e = upload_batch(m, X, nullptr, nullptr, n);
    if (e != cudaSuccess) return fail(e);
    forward(m, n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(Y, m->y, 4 * (size_t)n * m->nout, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GETT_OK : fail(e);
}
