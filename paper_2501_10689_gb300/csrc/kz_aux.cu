// Set-up kernels (step A0) and the adjoint contractions (step A10).
#include "kz_device.cuh"

namespace {

// Row k of the caller's packed H (vr_len[k] entries at in_off[k]) into the
// aligned layout [a_k, a_k + len2_k) at rptr[k], zero-filled outside the VR;
// optionally a BF16 (re, im) copy rounded to nearest even.
__global__ void pack_rows_kernel(const float2* __restrict__ Hin, const int* __restrict__ in_off,
                                 const int4* __restrict__ rows, const int* __restrict__ rptr, float2* Hc,
                                 __nv_bfloat162* Hb) {
    const int k = blockIdx.x;
    const int4 rd = rows[k];  // {a, len2, o, e}
    const int src = in_off[k], dst = rptr[k];
    for (int p = threadIdx.x; p < rd.y; p += blockDim.x) {
        const int n = rd.x + p;
        const float2 h = (n >= rd.z && n < rd.w) ? Hin[src + (n - rd.z)] : make_float2(0.f, 0.f);
        Hc[dst + p] = h;
        if (Hb) Hb[dst + p] = __float22bfloat162_rn(h);
    }
}

// ||h_k||^2 with FP64 accumulation (one block per row).
__global__ void row_norms_kernel(const float2* __restrict__ Hc, const int4* __restrict__ rows,
                                 const int* __restrict__ rptr, double* out_d, float* out_f) {
    __shared__ double part[32];
    const int k = blockIdx.x;
    const int4 rd = rows[k];
    const int base = rptr[k];
    double a = 0.0;
    for (int p = threadIdx.x; p < rd.y; p += blockDim.x) {
        const float2 h = Hc[base + p];
        a += (double)h.x * h.x + (double)h.y * h.y;
    }
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        out_d[k] = t;
        out_f[k] = (float)t;
    }
}

// Gt[:, j] = G_Q[:, j] + H G_X[:, j]   (one block per row, one warp per column).
__global__ void adjoint_rhs_kernel(const __grid_constant__ KzInst I, int nrhs, const float2* __restrict__ G_Q,
                                   const float2* __restrict__ G_X, float2* __restrict__ Gt) {
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int4 rd = I.rows[i];
    const int base = I.rptr[i];
    for (int j = warp; j < nrhs; j += nw) {
        const float2* g = G_X + (size_t)j * I.Nt;
        float ax = 0.f, ay = 0.f;
        for (int n = rd.z + lane; n < rd.w; n += 32) {
            const float2 h = I.Hc[base + (n - rd.x)];
            const float2 v = g[n];
            ax = fmaf(h.x, v.x, fmaf(-h.y, v.y, ax));
            ay = fmaf(h.x, v.y, fmaf(h.y, v.x, ay));
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if (lane == 0) {
            const float2 q = G_Q ? G_Q[(size_t)j * I.K + i] : make_float2(0.f, 0.f);
            Gt[(size_t)j * I.K + i] = make_float2(q.x + ax, q.y + ay);
        }
    }
}

// grad_H[k, n] = sum_j Q_kj conj(GX_nj) - Lam_kj conj(X_nj) - Q_kj conj(Y_nj) on row k's VR,
// written in the caller's packed layout (row k at in_off[k]).
__global__ void adjoint_grad_h_kernel(const __grid_constant__ KzInst I, int nrhs, const float2* __restrict__ Q,
                                      const float2* __restrict__ X, const float2* __restrict__ GX,
                                      const float2* __restrict__ Lam, const float2* __restrict__ Y,
                                      const int* __restrict__ in_off, float2* __restrict__ gH) {
    const int k = blockIdx.x;
    const int4 rd = I.rows[k];
    for (int n = rd.z + threadIdx.x; n < rd.w; n += blockDim.x) {
        float gx = 0.f, gy = 0.f;
        for (int j = 0; j < nrhs; ++j) {
            const float2 q = Q[(size_t)j * I.K + k];
            const float2 l = Lam[(size_t)j * I.K + k];
            const size_t o = (size_t)j * I.Nt + n;
            const float2 a = GX ? GX[o] : make_float2(0.f, 0.f);
            const float2 x = X[o];
            const float2 y = Y[o];
            // q conj(a - y) - l conj(x)
            const float2 c = make_float2(a.x - y.x, a.y - y.y);
            gx += q.x * c.x + q.y * c.y - (l.x * x.x + l.y * x.y);
            gy += q.y * c.x - q.x * c.y - (l.y * x.x - l.x * x.y);
        }
        gH[in_off[k] + (n - rd.z)] = make_float2(gx, gy);
    }
}

// grad_xi = -Re sum conj(Lam) Q  (single block, FP64 accumulation).
__global__ void adjoint_grad_xi_kernel(int count, const float2* __restrict__ Q, const float2* __restrict__ Lam,
                                       float* out) {
    __shared__ double part[32];
    double a = 0.0;
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
        const float2 q = Q[e], l = Lam[e];
        a += (double)l.x * q.x + (double)l.y * q.y;
    }
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *out = (float)(-t);
    }
}

// Batched forms: grid (item, row group); block y takes rows y, y + gridDim.y, ...
// of its item.
__global__ void adjoint_rhs_batched_kernel(const KzInst* __restrict__ insts, const KzAdjItem* __restrict__ adj,
                                           int nrhs) {
    const KzInst& I = insts[blockIdx.x];
    const KzAdjItem A = adj[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float2* Gt = const_cast<float2*>(I.s);
    for (int i = blockIdx.y; i < I.K; i += gridDim.y) {
        const int4 rd = I.rows[i];
        const int base = I.rptr[i];
        for (int j = warp; j < nrhs; j += nw) {
            float ax = 0.f, ay = 0.f;
            if (A.G_X) {
                const float2* g = A.G_X + (size_t)j * I.Nt;
                for (int n = rd.z + lane; n < rd.w; n += 32) {
                    const float2 h = I.Hc[base + (n - rd.x)];
                    const float2 v = g[n];
                    ax = fmaf(h.x, v.x, fmaf(-h.y, v.y, ax));
                    ay = fmaf(h.x, v.y, fmaf(h.y, v.x, ay));
                }
                ax = warp_sum(ax);
                ay = warp_sum(ay);
            }
            if (lane == 0) {
                const float2 q = A.G_Q ? A.G_Q[(size_t)j * I.K + i] : make_float2(0.f, 0.f);
                Gt[(size_t)j * I.K + i] = make_float2(q.x + ax, q.y + ay);
            }
        }
    }
}

// Lambda = I.v and Y = H^H Lambda = I.x are the adjoint batch's outputs.
__global__ void adjoint_grad_h_batched_kernel(const KzInst* __restrict__ insts, const KzAdjItem* __restrict__ adj,
                                              int nrhs) {
    const KzInst& I = insts[blockIdx.x];
    const KzAdjItem A = adj[blockIdx.x];
    const float2* Lam = I.v;
    const float2* Y = I.x;
    for (int k = blockIdx.y; k < I.K; k += gridDim.y) {
        const int4 rd = I.rows[k];
        for (int n = rd.z + threadIdx.x; n < rd.w; n += blockDim.x) {
            float gx = 0.f, gy = 0.f;
            for (int j = 0; j < nrhs; ++j) {
                const float2 q = A.Q[(size_t)j * I.K + k];
                const float2 l = Lam[(size_t)j * I.K + k];
                const size_t o = (size_t)j * I.Nt + n;
                const float2 a = A.G_X ? A.G_X[o] : make_float2(0.f, 0.f);
                const float2 x = A.X[o];
                const float2 y = Y[o];
                const float2 c = make_float2(a.x - y.x, a.y - y.y);
                gx += q.x * c.x + q.y * c.y - (l.x * x.x + l.y * x.y);
                gy += q.y * c.x - q.x * c.y - (l.y * x.x - l.x * x.y);
            }
            A.grad_H[I.in_off[k] + (n - rd.z)] = make_float2(gx, gy);
        }
    }
}

__global__ void adjoint_grad_xi_batched_kernel(const KzInst* __restrict__ insts, const KzAdjItem* __restrict__ adj,
                                               int nrhs) {
    __shared__ double part[32];
    const KzInst& I = insts[blockIdx.x];
    const KzAdjItem A = adj[blockIdx.x];
    const int count = I.K * nrhs;
    double a = 0.0;
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
        const float2 q = A.Q[e], l = I.v[e];
        a += (double)l.x * q.x + (double)l.y * q.y;
    }
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *A.grad_xi = (float)(-t);
    }
}

}  // namespace

cudaError_t kz_adjoint_rhs_batched(const KzInst* insts, const KzAdjItem* adj, int n, int K_max, int nrhs,
                                   cudaStream_t st) {
    adjoint_rhs_batched_kernel<<<dim3(n, std::min(K_max, 65535)), 256, 0, st>>>(insts, adj, nrhs);
    return cudaGetLastError();
}

cudaError_t kz_adjoint_contract_batched(const KzInst* insts, const KzAdjItem* adj, int n, int K_max, int nrhs,
                                        cudaStream_t st) {
    adjoint_grad_h_batched_kernel<<<dim3(n, std::min(K_max, 65535)), 256, 0, st>>>(insts, adj, nrhs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_grad_xi_batched_kernel<<<n, 1024, 0, st>>>(insts, adj, nrhs);
    return cudaGetLastError();
}

cudaError_t kz_pack_rows(const float2* Hin, const int* in_off, const int4* rows, const int* rptr, int K,
                         int64_t total2, float2* Hc, __nv_bfloat162* Hb, cudaStream_t st) {
    (void)total2;
    pack_rows_kernel<<<K, 256, 0, st>>>(Hin, in_off, rows, rptr, Hc, Hb);
    return cudaGetLastError();
}

cudaError_t kz_row_norms(const float2* Hc, const int4* rows, const int* rptr, int K, double* out_d, float* out_f,
                         cudaStream_t st) {
    row_norms_kernel<<<K, 256, 0, st>>>(Hc, rows, rptr, out_d, out_f);
    return cudaGetLastError();
}

cudaError_t kz_adjoint_rhs(const KzInst& I, int nrhs, const float2* G_Q, const float2* G_X, float2* Gt,
                           cudaStream_t st) {
    adjoint_rhs_kernel<<<I.K, 256, 0, st>>>(I, nrhs, G_Q, G_X, Gt);
    return cudaGetLastError();
}

cudaError_t kz_adjoint_contract(const KzInst& I, int nrhs, const float2* Q, const float2* X, const float2* G_X,
                                const float2* Lam, const float2* Y, const int* in_off, float2* grad_H,
                                float* grad_xi, cudaStream_t st) {
    adjoint_grad_h_kernel<<<I.K, 256, 0, st>>>(I, nrhs, Q, X, G_X, Lam, Y, in_off, grad_H);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adjoint_grad_xi_kernel<<<1, 1024, 0, st>>>(I.K * nrhs, Q, Lam, grad_xi);
    return cudaGetLastError();
}
