// Learned warm start: the encoder-decoder network behind hrt_net_* (include/hrt.h).
//
// Architecture (levels L, base width c, ch[l] = c 2^l): per encoder level two 3x3x3 conv+ReLU
// and a 2x average pool; a bottleneck of two conv+ReLU at ch[L]; per decoder level a 2x nearest
// upsample concatenated with the encoder skip and two conv+ReLU; a 1x1x1 head to one channel.
// Input: 2 feature channels (padded to 16); output: the normalised log10 temperature.
// Parameters are FP32 masters (Adam) with BF16 copies for the tensor-core kernels; activations
// and activation gradients are BF16, accumulation FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx_internal.h"
#include "nn.h"

using namespace hrt;
using hrt::nn::bf16;

namespace {

constexpr int CIN_REAL = 2;     // log density, log radiation flux
constexpr int CIN_PAD = 16;
// fixed feature / target normalisation
constexpr double F0_OFF = -21.5, F0_SCALE = 1.0;   // log10 rho [g/cm^3]
constexpr double F1_OFF = 0.0, F1_SCALE = 2.0;     // log10 F [erg/s/cm^2]
constexpr double T_OFF = 1.5, T_SCALE = 0.5;       // log10 T [K]

struct Layer {
    int cin, cin_real, cout;
    long long w_off, b_off;      // into the FP32 parameter vector
    bf16* wb = nullptr;          // [27][cin][cout]
    bf16* wt = nullptr;          // [27][cout][cin]
    bf16* wtp = nullptr;         // wt packed for the TMA-fed convolution (forward)
    bf16* wbp = nullptr;         // wb packed likewise (data gradient; null when cin % 32 != 0)
};

template <class T>
T* dalloc(size_t n, cudaError_t& e) {
    T* p = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    return p;
}

}  // namespace

struct hrt_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    int base = 32, levels = 2;
    std::vector<int> ch;
    std::vector<Layer> layers;   // encoder (2L), bottleneck (2), decoder (2L)
    long long head_w = 0, head_b = 0, nparam = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    int step = 0;
    // activations for one size
    int N = 0, D = 0, H = 0, W = 0;
    std::vector<void*> bufs;
    bf16* x_in = nullptr;
    std::vector<bf16*> e0, e1, pooled, ge0, ge1, gpooled;
    bf16 *b0 = nullptr, *b1 = nullptr, *gb0 = nullptr, *gb1 = nullptr;
    std::vector<bf16*> cat, d0, d1, gcat, gd0, gd1;
    float *y = nullptr, *dy = nullptr, *xf = nullptr, *tf = nullptr;
    double* loss = nullptr;
};

namespace {

#define NCK(call)                                 \
    do {                                          \
        cudaError_t _e = (call);                  \
        if (_e != cudaSuccess) {                  \
            cudaGetLastError();                   \
            return HRT_ECUDA;                     \
        }                                         \
    } while (0)

void free_acts(hrt_net* n) {
    for (void* b : n->bufs) cudaFree(b);
    n->bufs.clear();
    n->N = n->D = n->H = n->W = 0;
}

int alloc_acts(hrt_net* n, int N, int D, int H, int W) {
    if (n->N == N && n->D == D && n->H == H && n->W == W) return HRT_OK;
    free_acts(n);
    cudaError_t e = cudaSuccess;
    auto A = [&](size_t elems) {
        bf16* q = dalloc<bf16>(elems, e);
        n->bufs.push_back(q);
        return q;
    };
    const int L = n->levels;
    auto nv = [&](int l) { return (size_t)N * (D >> l) * (H >> l) * (W >> l); };
    n->x_in = A(nv(0) * CIN_PAD);
    n->e0.assign(L, nullptr); n->e1.assign(L, nullptr); n->pooled.assign(L, nullptr);
    n->ge0.assign(L, nullptr); n->ge1.assign(L, nullptr); n->gpooled.assign(L, nullptr);
    n->cat.assign(L, nullptr); n->d0.assign(L, nullptr); n->d1.assign(L, nullptr);
    n->gcat.assign(L, nullptr); n->gd0.assign(L, nullptr); n->gd1.assign(L, nullptr);
    for (int l = 0; l < L; ++l) {
        n->e0[l] = A(nv(l) * n->ch[l]); n->e1[l] = A(nv(l) * n->ch[l]);
        n->ge0[l] = A(nv(l) * n->ch[l]); n->ge1[l] = A(nv(l) * n->ch[l]);
        n->pooled[l] = A(nv(l + 1) * n->ch[l]); n->gpooled[l] = A(nv(l + 1) * n->ch[l]);
        const int cprev = n->ch[l + 1];
        n->cat[l] = A(nv(l) * (cprev + n->ch[l])); n->gcat[l] = A(nv(l) * (cprev + n->ch[l]));
        n->d0[l] = A(nv(l) * n->ch[l]); n->d1[l] = A(nv(l) * n->ch[l]);
        n->gd0[l] = A(nv(l) * n->ch[l]); n->gd1[l] = A(nv(l) * n->ch[l]);
    }
    n->b0 = A(nv(L) * n->ch[L]); n->b1 = A(nv(L) * n->ch[L]);
    n->gb0 = A(nv(L) * n->ch[L]); n->gb1 = A(nv(L) * n->ch[L]);
    float* f = dalloc<float>(nv(0) * 4 + nv(0) * CIN_REAL, e);
    n->bufs.push_back(f);
    n->y = f; n->dy = f + nv(0); n->tf = f + 2 * nv(0); n->xf = f + 4 * nv(0);
    n->loss = dalloc<double>(1, e);
    n->bufs.push_back(n->loss);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_acts(n);
        return e == cudaErrorMemoryAllocation ? HRT_ENOMEM : HRT_ECUDA;
    }
    n->N = N; n->D = D; n->H = H; n->W = W;
    return HRT_OK;
}

int refresh_bf16(hrt_net* n) {
    for (const Layer& l : n->layers) {
        NCK(nn::weights_bf16(n->p + l.w_off, l.wb, l.wt, l.cin, l.cin, l.cout, n->stream));
        NCK(nn::pack_tma_weights(l.wt, l.wtp, l.cin, l.cout, n->stream));
        if (l.wbp) NCK(nn::pack_tma_weights(l.wb, l.wbp, l.cout, l.cin, n->stream));
    }
    return HRT_OK;
}

// forward pass; inputs in n->xf (float [NV][2]); output n->y (float [NV])
int forward(hrt_net* n) {
    const cudaStream_t s = n->stream;
    const int L = n->levels, N = n->N;
    NCK(nn::pack_input(n->xf, n->x_in, (long long)N * n->D * n->H * n->W, CIN_REAL, CIN_PAD, s));
    const bf16* h = n->x_in;
    int k = 0;
    for (int l = 0; l < L; ++l) {
        const int D = n->D >> l, H = n->H >> l, W = n->W >> l;
        const Layer& a = n->layers[k++];
        NCK(nn::conv3d(h, a.wt, a.wtp, n->p + a.b_off, n->e0[l], N, D, H, W, a.cin, a.cout, false, true, s));
        const Layer& b = n->layers[k++];
        NCK(nn::conv3d(n->e0[l], b.wt, b.wtp, n->p + b.b_off, n->e1[l], N, D, H, W, b.cin, b.cout, false, true, s));
        NCK(nn::pool2(n->e1[l], n->pooled[l], N, D, H, W, n->ch[l], s));
        h = n->pooled[l];
    }
    {
        const int D = n->D >> L, H = n->H >> L, W = n->W >> L;
        const Layer& a = n->layers[k++];
        NCK(nn::conv3d(h, a.wt, a.wtp, n->p + a.b_off, n->b0, N, D, H, W, a.cin, a.cout, false, true, s));
        const Layer& b = n->layers[k++];
        NCK(nn::conv3d(n->b0, b.wt, b.wtp, n->p + b.b_off, n->b1, N, D, H, W, b.cin, b.cout, false, true, s));
        h = n->b1;
    }
    for (int l = L - 1; l >= 0; --l) {
        const int D = n->D >> l, H = n->H >> l, W = n->W >> l;
        const int cprev = n->ch[l + 1];
        NCK(nn::concat_up(h, n->e1[l], n->cat[l], N, D, H, W, cprev, n->ch[l], s));
        const Layer& a = n->layers[k++];
        NCK(nn::conv3d(n->cat[l], a.wt, a.wtp, n->p + a.b_off, n->d0[l], N, D, H, W, a.cin, a.cout, false, true, s));
        const Layer& b = n->layers[k++];
        NCK(nn::conv3d(n->d0[l], b.wt, b.wtp, n->p + b.b_off, n->d1[l], N, D, H, W, b.cin, b.cout, false, true, s));
        h = n->d1[l];
    }
    NCK(nn::head_forward(h, n->p + n->head_w, n->p + n->head_b, n->y, (long long)N * n->D * n->H * n->W, n->ch[0], s));
    return HRT_OK;
}

// one conv layer backward: g is dL/d(output after ReLU) (masked in place), in the layer input;
// writes dW, db into n->g and, if gin, dL/d(input)
int conv_back(hrt_net* n, const Layer& ly, const bf16* in, const bf16* out, bf16* g, bf16* gin, int D, int H, int W) {
    const cudaStream_t s = n->stream;
    const long long NV = (long long)n->N * D * H * W;
    NCK(nn::relu_mask(g, out, NV * ly.cout, s));
    NCK(nn::conv3d_wgrad(in, g, n->g + ly.w_off, n->N, D, H, W, ly.cin, ly.cout, s));
    NCK(nn::bias_grad(g, n->g + ly.b_off, NV, ly.cout, s));
    if (gin) NCK(nn::conv3d(g, ly.wb, ly.wbp, nullptr, gin, n->N, D, H, W, ly.cout, ly.cin, true, false, s));
    return HRT_OK;
}

// backward pass after forward(); loss gradient in n->dy; accumulates into n->g
int backward(hrt_net* n) {
    const cudaStream_t s = n->stream;
    const int L = n->levels, N = n->N;
    const long long NV0 = (long long)N * n->D * n->H * n->W;
    NCK(nn::head_backward(n->d1[0], n->p + n->head_w, n->dy, n->gd1[0], n->g + n->head_w, n->g + n->head_b, NV0,
                          n->ch[0], s));
    int k = (int)n->layers.size() - 1;
    for (int l = 0; l < L; ++l) {          // decoder, last level first
        const int D = n->D >> l, H = n->H >> l, W = n->W >> l;
        const long long NV = (long long)N * D * H * W;
        const Layer& b = n->layers[k--];
        const Layer& a = n->layers[k--];
        int rc = conv_back(n, b, n->d0[l], n->d1[l], n->gd1[l], n->gd0[l], D, H, W);
        if (rc != HRT_OK) return rc;
        rc = conv_back(n, a, n->cat[l], n->d0[l], n->gd0[l], n->gcat[l], D, H, W);
        if (rc != HRT_OK) return rc;
        bf16* glow = (l + 1 < L) ? n->gd1[l + 1] : n->gb1;
        NCK(cudaMemsetAsync(n->ge1[l], 0, NV * n->ch[l] * sizeof(bf16), s));
        NCK(nn::concat_up_back(n->gcat[l], glow, n->ge1[l], N, D, H, W, n->ch[l + 1], n->ch[l], s));
    }
    {
        const int D = n->D >> L, H = n->H >> L, W = n->W >> L;
        const Layer& b = n->layers[k--];
        const Layer& a = n->layers[k--];
        int rc = conv_back(n, b, n->b0, n->b1, n->gb1, n->gb0, D, H, W);
        if (rc != HRT_OK) return rc;
        rc = conv_back(n, a, n->pooled[L - 1], n->b0, n->gb0, n->gpooled[L - 1], D, H, W);
        if (rc != HRT_OK) return rc;
    }
    for (int l = L - 1; l >= 0; --l) {     // encoder
        const int D = n->D >> l, H = n->H >> l, W = n->W >> l;
        NCK(nn::pool2_back(n->gpooled[l], n->ge1[l], N, D, H, W, n->ch[l], true, s));
        const Layer& b = n->layers[k--];
        const Layer& a = n->layers[k--];
        int rc = conv_back(n, b, n->e0[l], n->e1[l], n->ge1[l], n->ge0[l], D, H, W);
        if (rc != HRT_OK) return rc;
        const bf16* in = l == 0 ? n->x_in : n->pooled[l - 1];
        rc = conv_back(n, a, in, n->e0[l], n->ge0[l], l == 0 ? nullptr : n->gpooled[l - 1], D, H, W);
        if (rc != HRT_OK) return rc;
    }
    return HRT_OK;
}

bool dims_ok(const hrt_net* n, int N, int D, int H, int W) {
    const int m = 1 << n->levels;
    return N >= 1 && D >= m && H >= m && W >= m && D % m == 0 && H % m == 0 && W % m == 0;
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// parameter vector <-> the packed layout [27][cin_real][cout], b[cout] per layer, head w, b
long long packed_count(const hrt_net* n) {
    long long c = 0;
    for (const Layer& l : n->layers) c += 27LL * l.cin_real * l.cout + l.cout;
    return c + n->ch[0] + 1;
}

// features of a Cartesian context: normalised log10 rho and log10 of the summed point-source flux
__global__ void k_features(DevGrid g, DevSources s, const double* srcL, double L0, float* out) {
    const long long nc = g.ncells;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c % g.n1), j = (int)((c / g.n1) % g.n2), k = (int)(c / ((long long)g.n1 * g.n2));
        const double x = 0.5 * ((double)g.w1[i] + g.w1[i + 1]), y = 0.5 * ((double)g.w2[j] + g.w2[j + 1]),
                     z = 0.5 * ((double)g.w3[k] + g.w3[k + 1]);
        const double hw = 0.5 * ((double)g.w1[i + 1] - g.w1[i]);
        double F = 0.0;
        for (int q = 0; q < s.npoint; ++q) {
            const double dx = x - s.pos[3 * q], dy = y - s.pos[3 * q + 1], dz = z - s.pos[3 * q + 2];
            F += srcL[q] / (4.0 * 3.14159265358979323846 * ((dx * dx + dy * dy + dz * dz + hw * hw) * L0 * L0));
        }
        const double rho = (double)g.rhoL[c] / L0;
        out[2 * c] = (float)((log10(rho > 1e-300 ? rho : 1e-300) - F0_OFF) / F0_SCALE);
        out[2 * c + 1] = (float)((log10(F > 1e-300 ? F : 1e-300) - F1_OFF) / F1_SCALE);
    }
}

__global__ void k_to_temperature(const float* y, double* T, long long n, double tmin, double tmax) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
        const double t = pow(10.0, T_OFF + T_SCALE * (double)y[c]);
        T[c] = t < tmin ? tmin : (t > tmax ? tmax : t);
    }
}

__global__ void k_from_temperature(const double* T, float* y, long long n) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x)
        y[c] = (float)((log10(T[c]) - T_OFF) / T_SCALE);
}

}  // namespace

extern "C" {

static int net_create(hrt_net** out, int device, const int* widths, int levels, uint64_t seed, void* stream) {
    *out = nullptr;
    hrt_net* n = new hrt_net();
    n->device = device;
    n->stream = (cudaStream_t)stream;
    n->base = widths[0];
    n->levels = levels;
    Guard gd(device);
    for (int l = 0; l <= levels; ++l) n->ch.push_back(widths[l]);
    long long off = 0;
    auto add = [&](int cin_real, int cin, int cout) {
        Layer ly;
        ly.cin = cin; ly.cin_real = cin_real; ly.cout = cout;
        ly.w_off = off; off += 27LL * cin * cout;
        ly.b_off = off; off += cout;
        n->layers.push_back(ly);
    };
    int c = CIN_PAD;
    for (int l = 0; l < levels; ++l) {
        add(l == 0 ? CIN_REAL : c, c, n->ch[l]);
        add(n->ch[l], n->ch[l], n->ch[l]);
        c = n->ch[l];
    }
    add(c, c, n->ch[levels]);
    add(n->ch[levels], n->ch[levels], n->ch[levels]);
    c = n->ch[levels];
    for (int l = levels - 1; l >= 0; --l) {
        add(c + n->ch[l], c + n->ch[l], n->ch[l]);
        add(n->ch[l], n->ch[l], n->ch[l]);
        c = n->ch[l];
    }
    n->head_w = off; off += n->ch[0];
    n->head_b = off; off += 1;
    n->nparam = off;
    cudaError_t e = cudaSuccess;
    n->p = dalloc<float>(off, e); n->g = dalloc<float>(off, e);
    n->m = dalloc<float>(off, e); n->v = dalloc<float>(off, e);
    for (Layer& ly : n->layers) {
        ly.wb = dalloc<bf16>(27LL * ly.cin * ly.cout, e);
        ly.wt = dalloc<bf16>(27LL * ly.cin * ly.cout, e);
        ly.wtp = dalloc<bf16>(27LL * ly.cin * ly.cout, e);
        if (ly.cin % 32 == 0) ly.wbp = dalloc<bf16>(27LL * ly.cin * ly.cout, e);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        hrt_net_destroy(n);
        return HRT_ENOMEM;
    }
    cudaMemsetAsync(n->p, 0, off * sizeof(float), n->stream);
    cudaMemsetAsync(n->m, 0, off * sizeof(float), n->stream);
    cudaMemsetAsync(n->v, 0, off * sizeof(float), n->stream);
    // Kaiming-uniform weights (padded input channels of the first layer stay zero), zero biases
    unsigned long long sd = seed;
    for (const Layer& ly : n->layers) {
        const float bound = sqrtf(6.f / (27.f * ly.cin_real));
        if (ly.cin == ly.cin_real) {
            nn::init_uniform(n->p + ly.w_off, 27LL * ly.cin * ly.cout, bound, ++sd, n->stream);
        } else {
            for (int t = 0; t < 27; ++t)
                nn::init_uniform(n->p + ly.w_off + (long long)t * ly.cin * ly.cout, (long long)ly.cin_real * ly.cout,
                                 bound, ++sd * 1000003ull + t, n->stream);
        }
    }
    nn::init_uniform(n->p + n->head_w, n->ch[0], 1.f / sqrtf((float)n->ch[0]), ++sd, n->stream);
    if (refresh_bf16(n) != HRT_OK || cudaStreamSynchronize(n->stream) != cudaSuccess) {
        cudaGetLastError();
        hrt_net_destroy(n);
        return HRT_ECUDA;
    }
    *out = n;
    return HRT_OK;
}

int hrt_net_create(hrt_net** out, int device, int base_channels, int levels, uint64_t seed, void* stream) {
    if (!out || base_channels < 32 || base_channels % 32 != 0 || levels < 1 || levels > 4) return HRT_EINVAL;
    int w[5];
    for (int l = 0; l <= levels; ++l) w[l] = base_channels << l;
    return net_create(out, device, w, levels, seed, stream);
}

int hrt_net_create_widths(hrt_net** out, int device, const int* widths, int levels, uint64_t seed, void* stream) {
    if (!out || !widths || levels < 1 || levels > 4) return HRT_EINVAL;
    for (int l = 0; l <= levels; ++l)
        if (widths[l] < 32 || widths[l] % 32 != 0 || widths[l] > 512) return HRT_EINVAL;
    return net_create(out, device, widths, levels, seed, stream);
}

int hrt_net_destroy(hrt_net* n) {
    if (!n) return HRT_EINVAL;
    Guard gd(n->device);
    cudaStreamSynchronize(n->stream);
    free_acts(n);
    for (Layer& ly : n->layers) {
        for (bf16* q : {ly.wb, ly.wt, ly.wtp, ly.wbp})
            if (q) cudaFree(q);
    }
    for (float* q : {n->p, n->g, n->m, n->v})
        if (q) cudaFree(q);
    delete n;
    return HRT_OK;
}

int64_t hrt_net_num_params(const hrt_net* n) { return n ? packed_count(n) : -1; }

int hrt_net_get_params(hrt_net* n, float* out, int64_t count) {
    if (!n || !out || count < packed_count(n)) return HRT_EINVAL;
    Guard gd(n->device);
    std::vector<float> all(n->nparam);
    NCK(cudaMemcpyAsync(all.data(), n->p, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    long long q = 0;
    for (const Layer& ly : n->layers) {
        for (int t = 0; t < 27; ++t)
            for (int i = 0; i < ly.cin_real; ++i)
                for (int o = 0; o < ly.cout; ++o) out[q++] = all[ly.w_off + ((long long)t * ly.cin + i) * ly.cout + o];
        for (int o = 0; o < ly.cout; ++o) out[q++] = all[ly.b_off + o];
    }
    for (int c = 0; c < n->ch[0]; ++c) out[q++] = all[n->head_w + c];
    out[q++] = all[n->head_b];
    return HRT_OK;
}

int hrt_net_set_params(hrt_net* n, const float* in, int64_t count) {
    if (!n || !in || count < packed_count(n)) return HRT_EINVAL;
    Guard gd(n->device);
    std::vector<float> all(n->nparam, 0.f);
    long long q = 0;
    for (const Layer& ly : n->layers) {
        for (int t = 0; t < 27; ++t)
            for (int i = 0; i < ly.cin_real; ++i)
                for (int o = 0; o < ly.cout; ++o) all[ly.w_off + ((long long)t * ly.cin + i) * ly.cout + o] = in[q++];
        for (int o = 0; o < ly.cout; ++o) all[ly.b_off + o] = in[q++];
    }
    for (int c = 0; c < n->ch[0]; ++c) all[n->head_w + c] = in[q++];
    all[n->head_b] = in[q++];
    NCK(cudaMemcpyAsync(n->p, all.data(), n->nparam * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    NCK(cudaMemsetAsync(n->m, 0, n->nparam * sizeof(float), n->stream));
    NCK(cudaMemsetAsync(n->v, 0, n->nparam * sizeof(float), n->stream));
    n->step = 0;
    const int rc = refresh_bf16(n);
    if (rc != HRT_OK) return rc;
    NCK(cudaStreamSynchronize(n->stream));
    return HRT_OK;
}

int hrt_net_forward(hrt_net* n, int N, int D, int H, int W, const float* d_in, float* d_out) {
    if (!n || !d_in || !d_out || !dims_ok(n, N, D, H, W)) return HRT_EINVAL;
    Guard gd(n->device);
    int rc = alloc_acts(n, N, D, H, W);
    if (rc != HRT_OK) return rc;
    const long long NV = (long long)N * D * H * W;
    NCK(cudaMemcpyAsync(n->xf, d_in, NV * CIN_REAL * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    rc = forward(n);
    if (rc != HRT_OK) return rc;
    NCK(cudaMemcpyAsync(d_out, n->y, NV * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    int failed = 0;
    NCK(nn::tc_status(&failed, n->stream));     // synchronises the stream
    return failed ? HRT_ETIMEDOUT : HRT_OK;
}

static int grad_pass(hrt_net* n, int N, int D, int H, int W, const float* d_in, const float* d_target, double* loss_out) {
    if (!n || !d_in || !d_target || !dims_ok(n, N, D, H, W)) return HRT_EINVAL;
    int rc = alloc_acts(n, N, D, H, W);
    if (rc != HRT_OK) return rc;
    const long long NV = (long long)N * D * H * W;
    NCK(cudaMemcpyAsync(n->xf, d_in, NV * CIN_REAL * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    NCK(cudaMemcpyAsync(n->tf, d_target, NV * sizeof(float), cudaMemcpyDeviceToDevice, n->stream));
    NCK(cudaMemsetAsync(n->g, 0, n->nparam * sizeof(float), n->stream));
    NCK(cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
    rc = forward(n);
    if (rc != HRT_OK) return rc;
    NCK(nn::mse_loss(n->y, n->tf, n->dy, n->loss, NV, n->stream));
    rc = backward(n);
    if (rc != HRT_OK) return rc;
    // a tensor-core wait that gave up leaves the gradients invalid: no step is taken on them
    int failed = 0;
    NCK(nn::tc_status(&failed, n->stream));
    if (failed) return HRT_ETIMEDOUT;
    if (loss_out) {
        NCK(cudaMemcpyAsync(loss_out, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        NCK(cudaStreamSynchronize(n->stream));
    }
    return HRT_OK;
}

int hrt_net_gradients(hrt_net* n, int N, int D, int H, int W, const float* d_in, const float* d_target, float* grad,
                      int64_t count, double* loss_out) {
    if (!n || !grad || count < packed_count(n)) return HRT_EINVAL;
    Guard gd(n->device);
    int rc = grad_pass(n, N, D, H, W, d_in, d_target, loss_out);
    if (rc != HRT_OK) return rc;
    std::vector<float> all(n->nparam);
    NCK(cudaMemcpyAsync(all.data(), n->g, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(cudaStreamSynchronize(n->stream));
    long long q = 0;
    for (const Layer& ly : n->layers) {
        for (int t = 0; t < 27; ++t)
            for (int i = 0; i < ly.cin_real; ++i)
                for (int o = 0; o < ly.cout; ++o) grad[q++] = all[ly.w_off + ((long long)t * ly.cin + i) * ly.cout + o];
        for (int o = 0; o < ly.cout; ++o) grad[q++] = all[ly.b_off + o];
    }
    for (int c = 0; c < n->ch[0]; ++c) grad[q++] = all[n->head_w + c];
    grad[q++] = all[n->head_b];
    return HRT_OK;
}

int hrt_net_train_step(hrt_net* n, int N, int D, int H, int W, const float* d_in, const float* d_target, float lr,
                       double* loss_out) {
    if (!n || !(lr > 0)) return HRT_EINVAL;
    Guard gd(n->device);
    int rc = grad_pass(n, N, D, H, W, d_in, d_target, nullptr);
    if (rc != HRT_OK) return rc;
    n->step += 1;
    NCK(nn::adam(n->p, n->g, n->m, n->v, n->nparam, lr, n->step, n->stream));
    rc = refresh_bf16(n);
    if (rc != HRT_OK) return rc;
    if (loss_out) {
        NCK(cudaMemcpyAsync(loss_out, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        NCK(cudaStreamSynchronize(n->stream));
    }
    return HRT_OK;
}

int hrt_net_features(hrt_ctx* ctx, float* d_out, int64_t n) {
    if (!ctx || !d_out) return HRT_EINVAL;
    if (ctx->gtype != GRID_CARTESIAN) return ctx->fail(HRT_EINVAL, "features need a Cartesian grid");
    if (n < 2 * ctx->ncells()) return ctx->fail(HRT_EINVAL, "features need 2 floats per cell");
    int rc = prepare_ctx(ctx);
    if (rc != HRT_OK) return rc;
    Guard gd(ctx->device);
    std::vector<double> L(std::max<size_t>(ctx->pts.size(), 1), 0.0);
    for (size_t q = 0; q < ctx->pts.size(); ++q) L[q] = ctx->pts[q].L;
    double* dL = nullptr;
    CK(cudaMalloc(&dL, L.size() * sizeof(double)), "features");
    cudaMemcpyAsync(dL, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    k_features<<<512, 256, 0, ctx->stream>>>(ctx->grid, ctx->src, dL, ctx->L0, d_out);
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dL);
    CK(e, "features");
    return HRT_OK;
}

int hrt_net_temperature_target(hrt_ctx* ctx, float* d_out, int64_t n) {
    if (!ctx || !d_out || n < ctx->ncells() || !ctx->d_T.p) return HRT_EINVAL;
    Guard gd(ctx->device);
    k_from_temperature<<<512, 256, 0, ctx->stream>>>(ctx->d_T.p, d_out, ctx->ncells());
    CK(cudaStreamSynchronize(ctx->stream), "target");
    return HRT_OK;
}

int hrt_net_warm_start(hrt_net* n, hrt_ctx* ctx) {
    if (!n || !ctx) return HRT_EINVAL;
    if (ctx->gtype != GRID_CARTESIAN) return ctx->fail(HRT_EINVAL, "warm start needs a Cartesian grid");
    const int nx = ctx->n[0], ny = ctx->n[1], nz = ctx->n[2];
    if (!dims_ok(n, 1, nz, ny, nx)) return ctx->fail(HRT_EINVAL, "grid dims must be multiples of 2^levels");
    Guard gd(n->device);
    int rc = alloc_acts(n, 1, nz, ny, nx);
    if (rc != HRT_OK) return rc;
    rc = hrt_net_features(ctx, n->xf, 2 * ctx->ncells());
    if (rc != HRT_OK) return rc;
    const cudaStream_t keep = n->stream;
    n->stream = ctx->stream;
    rc = forward(n);
    n->stream = keep;
    if (rc != HRT_OK) return rc;
    int failed = 0;
    CK(nn::tc_status(&failed, ctx->stream), "warm start");
    if (failed) return ctx->fail(HRT_ETIMEDOUT, "a tensor-core wait gave up; the temperatures are unchanged");
    k_to_temperature<<<512, 256, 0, ctx->stream>>>(n->y, ctx->d_T.p, ctx->ncells(), ctx->Tn.front(), ctx->Tn.back());
    CK(cudaStreamSynchronize(ctx->stream), "warm start");
    ctx->have_T = true;
    return HRT_OK;
}

// ---------------------------------------------------------------- single-layer hooks
// which kernel a hook runs: the TMA-fed pipeline, the per-phase tcgen05 kernel, or mma.sync
enum ConvImpl { CONV_TMA = 0, CONV_PHASED = 1, CONV_MMA = 2 };
static int conv3d_hook(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                       const float* d_b, int relu, float* d_y, void* stream, int impl);

int hrt_nn_conv3d(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w, const float* d_b,
                  int relu, float* d_y, void* stream) {
    return conv3d_hook(N, D, H, W, Cin, Cout, d_x, d_w, d_b, relu, d_y, stream, CONV_TMA);
}

int hrt_nn_conv3d_phased(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                         const float* d_b, int relu, float* d_y, void* stream) {
    return conv3d_hook(N, D, H, W, Cin, Cout, d_x, d_w, d_b, relu, d_y, stream, CONV_PHASED);
}

int hrt_nn_conv3d_mma(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                      const float* d_b, int relu, float* d_y, void* stream) {
    return conv3d_hook(N, D, H, W, Cin, Cout, d_x, d_w, d_b, relu, d_y, stream, CONV_MMA);
}

static int conv3d_hook(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                       const float* d_b, int relu, float* d_y, void* stream, int impl) {
    if (N < 1 || D < 1 || H < 1 || W < 1 || Cin % 16 || Cout % 32 || !d_x || !d_w || !d_y) return HRT_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    const long long NV = (long long)N * D * H * W;
    cudaError_t e = cudaSuccess;
    bf16* x = dalloc<bf16>(NV * Cin, e);
    bf16* y = dalloc<bf16>(NV * Cout, e);
    bf16* wb = dalloc<bf16>(27LL * Cin * Cout, e);
    bf16* wt = dalloc<bf16>(27LL * Cin * Cout, e);
    bf16* wtp = dalloc<bf16>(27LL * Cin * Cout, e);
    if (e == cudaSuccess) e = nn::f32_to_bf16(d_x, x, NV * Cin, s);
    if (e == cudaSuccess) e = nn::weights_bf16(d_w, wb, wt, Cin, Cin, Cout, s);
    if (e == cudaSuccess) e = nn::pack_tma_weights(wt, wtp, Cin, Cout, s);
    if (e == cudaSuccess)
        e = impl == CONV_MMA      ? nn::conv3d_mma(x, wt, d_b, y, N, D, H, W, Cin, Cout, false, relu != 0, s)
            : impl == CONV_PHASED ? nn::conv3d_phased(x, wt, d_b, y, N, D, H, W, Cin, Cout, false, relu != 0, s)
                                  : nn::conv3d(x, wt, wtp, d_b, y, N, D, H, W, Cin, Cout, false, relu != 0, s);
    if (e == cudaSuccess) e = nn::bf16_to_f32(y, d_y, NV * Cout, s);
    int failed = 0;
    if (e == cudaSuccess) e = nn::tc_status(&failed, s);
    cudaFree(x); cudaFree(y); cudaFree(wb); cudaFree(wt); cudaFree(wtp);
    if (e != cudaSuccess) cudaGetLastError();
    if (e == cudaSuccess && failed) return HRT_ETIMEDOUT;
    return e == cudaSuccess ? HRT_OK : HRT_ECUDA;
}

int hrt_nn_conv3d_backward(int N, int D, int H, int W, int Cin, int Cout, const float* d_x, const float* d_w,
                           const float* d_dy, float* d_dx, float* d_dw, float* d_db, void* stream) {
    if (N < 1 || D < 1 || H < 1 || W < 1 || Cin % 32 || Cout % 32 || !d_x || !d_w || !d_dy || !d_dx || !d_dw || !d_db)
        return HRT_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    const long long NV = (long long)N * D * H * W;
    cudaError_t e = cudaSuccess;
    bf16* x = dalloc<bf16>(NV * Cin, e);
    bf16* g = dalloc<bf16>(NV * Cout, e);
    bf16* gx = dalloc<bf16>(NV * Cin, e);
    bf16* wb = dalloc<bf16>(27LL * Cin * Cout, e);
    bf16* wt = dalloc<bf16>(27LL * Cin * Cout, e);
    bf16* wbp = dalloc<bf16>(27LL * Cin * Cout, e);
    if (e == cudaSuccess) e = nn::f32_to_bf16(d_x, x, NV * Cin, s);
    if (e == cudaSuccess) e = nn::f32_to_bf16(d_dy, g, NV * Cout, s);
    if (e == cudaSuccess) e = nn::weights_bf16(d_w, wb, wt, Cin, Cin, Cout, s);
    if (e == cudaSuccess) e = nn::pack_tma_weights(wb, wbp, Cout, Cin, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_dw, 0, 27LL * Cin * Cout * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_db, 0, Cout * sizeof(float), s);
    if (e == cudaSuccess) e = nn::conv3d_wgrad(x, g, d_dw, N, D, H, W, Cin, Cout, s);
    if (e == cudaSuccess) e = nn::bias_grad(g, d_db, NV, Cout, s);
    if (e == cudaSuccess) e = nn::conv3d(g, wb, wbp, nullptr, gx, N, D, H, W, Cout, Cin, true, false, s);
    if (e == cudaSuccess) e = nn::bf16_to_f32(gx, d_dx, NV * Cin, s);
    int failed = 0;
    if (e == cudaSuccess) e = nn::tc_status(&failed, s);
    cudaFree(x); cudaFree(g); cudaFree(gx); cudaFree(wb); cudaFree(wt); cudaFree(wbp);
    if (e != cudaSuccess) cudaGetLastError();
    if (e == cudaSuccess && failed) return HRT_ETIMEDOUT;
    return e == cudaSuccess ? HRT_OK : HRT_ECUDA;
}

}  // extern "C"
