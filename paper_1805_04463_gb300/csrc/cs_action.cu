// cs_action.cu -- Benincasa-Dowker action from the interval abundances
// (Section "The Benincasa-Dowker Action": Eqs. s2d_local, s3d_local,
// s4d_local, the smeared actions and the smearing functions f2, f3, f4).
//
// The local action is an exact integer bracket times a constant.  The
// smeared action sums N_k f(k, eps) over the whole histogram; those terms are
// orders of magnitude larger than the result (the thesis notes this for its
// de Sitter runs), so every term and the sum are carried in double-double
// arithmetic (FP64 error-free transformations), which keeps the cancellation
// far below a 1e-12 relative error at the largest N.
#include <cmath>

#include "cs_action.cuh"
#include "cs_kernels.cuh"

namespace cs {

namespace {

__global__ void __launch_bounds__(kActThreads) k_action_partial(int dim, int64_t n, const int64_t* __restrict__ hist,
                                                                int64_t len, EpsArgs eps, dd* __restrict__ partial) {
    __shared__ dd red[kActThreads];
    const int tid = threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * kActThreads;
    for (int e = 0; e < eps.n; ++e) {
        const double ep = eps.v[e];
        if (is_local(ep)) continue;  // uniform across the grid
        const dd q = dd_two_sum(1.0, -ep);
        const int64_t kend = eps.kend[e];
        dd sum = dd_from(0.0);
        for (int64_t k = blockIdx.x * int64_t(kActThreads) + tid; k < kend; k += stride) {
            const int64_t hk = hist[k];
            if (hk == 0) continue;
            const dd f = dd_mul(dd_pow(q, smear_qexp(dim, k)), smear_poly(dim, k, q, ep));
            sum = dd_add(sum, dd_mul(dd_from_i64(hk), f));
        }
        red[tid] = sum;
        __syncthreads();
        for (int s = kActThreads / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] = dd_add(red[tid], red[tid + s]);
            __syncthreads();
        }
        if (tid == 0) partial[blockIdx.x * kMaxEps + e] = red[0];
        __syncthreads();
    }
}

__global__ void k_action_final(int dim, int64_t n, const int64_t* __restrict__ hist, int64_t len, EpsArgs eps,
                               const dd* __restrict__ partial, int nblocks, double* __restrict__ out,
                               int64_t* __restrict__ bracket) {
    const int e = threadIdx.x;
    int64_t h4[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4 && k < len; ++k) h4[k] = hist[k];
    const int64_t b = bracket_of(dim, n, h4);
    if (e == 0 && bracket) *bracket = b;
    if (e >= eps.n) return;
    const double ep = eps.v[e];
    dd s;
    if (is_local(ep)) {
        s = local_action(dim, b);
    } else {
        dd sum = dd_from(0.0);
        for (int blk = 0; blk < nblocks; ++blk) sum = dd_add(sum, partial[blk * kMaxEps + e]);
        s = smeared_action(dim, n, ep, sum);
    }
    out[e] = s.hi + s.lo;
}

// B phi(j) from the layer sums (Eqs. b2d_local, b3d_local, b4d_local), one
// thread per element.
__global__ void k_dalembertian(int dim, int64_t n, const double* __restrict__ phi, const double* __restrict__ layer,
                               double scale, double* __restrict__ out) {
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        const double p = phi ? phi[j] : 1.0;
        const double s0 = layer[j], s1 = layer[n + j], s2 = layer[2 * n + j];
        double b;
        if (dim == 2) {
            b = -p + 2.0 * (s0 - 2.0 * s1 + s2);
        } else if (dim == 3) {
            b = -p + s0 - 3.375 * s1 + 2.25 * s2;
        } else {
            const double s3 = layer[3 * n + j];
            b = -p + s0 - 9.0 * s1 + 16.0 * s2 - 8.0 * s3;
        }
        out[j] = scale * b;
    }
}

}  // namespace

cudaError_t launch_dalembertian(int dim, int64_t n, const double* phi, const double* layer, double ell, double* out,
                                cudaStream_t st) {
    const dd l2 = dd_two_prod(ell, ell);
    const dd c = dim == 2   ? dd_div(dd_from(2.0), l2)
                 : dim == 3 ? dd_div(dd_from(c3_const()), l2)
                            : dd_div(dd_from(4.0), dd_mul(l2, dd_sqrt(dd_from(6.0))));
    int64_t g = (n + 255) / 256;
    if (g > int64_t(device_sm_count()) * 8) g = int64_t(device_sm_count()) * 8;
    if (g < 1) g = 1;
    k_dalembertian<<<unsigned(g), 256, 0, st>>>(dim, n, phi, layer, c.hi + c.lo, out);
    return cudaGetLastError();
}

size_t action_workspace_bytes() { return sizeof(WsHeader) + size_t(kActBlocks) * kMaxEps * sizeof(dd); }

int action_host(int dim, int64_t n, const int64_t* hist, int64_t len, double eps, double* out, int64_t* bracket) {
    if (dim < 2 || dim > 4 || n < 0 || len < 0 || !(eps <= 1.0) || (len > 0 && !hist)) return CS_EINVAL;
    int64_t h4[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4 && k < len; ++k) h4[k] = hist[k];
    const int64_t b = bracket_of(dim, n, h4);
    if (bracket) *bracket = b;
    dd s;
    if (is_local(eps)) {
        s = local_action(dim, b);
    } else {
        const dd q = dd_two_sum(1.0, -eps);
        double R = 0.0;  // any histogram may come in here: bound by its own sum
        for (int64_t k = 0; k < len; ++k) R += fabs(double(hist[k]));
        const int64_t kend = smear_cutoff(dim, eps, R, len);
        dd sum = dd_from(0.0), p = dd_from(1.0);  // p = q^(max(0, k - deg))
        const int64_t deg = smear_deg(dim);
        for (int64_t k = 0; k < kend; ++k) {
            if (hist[k] != 0) sum = dd_add(sum, dd_mul(dd_from_i64(hist[k]), dd_mul(p, smear_poly(dim, k, q, eps))));
            if (k >= deg) p = dd_mul(p, q);
        }
        s = smeared_action(dim, n, eps, sum);
    }
    if (out) *out = s.hi + s.lo;
    return CS_OK;
}

cudaError_t launch_action_device(int dim, int64_t n, const int64_t* hist, int64_t len, const double* eps, int n_eps,
                                 double* out, int64_t* bracket, void* workspace, cudaStream_t st) {
    EpsArgs a;
    a.n = n_eps;
    bool any_smeared = false;
    for (int e = 0; e < kMaxEps; ++e) {
        a.v[e] = e < n_eps ? eps[e] : 0.0;
        a.kend[e] = is_local(a.v[e]) ? 0 : smear_cutoff(dim, a.v[e], 0.5 * double(n) * double(n), len);
        if (e < n_eps && !is_local(a.v[e])) any_smeared = true;
    }
    // Blocks that hold terms only: block b's threads take k = 256 b + t (one
    // term each while the grid covers the longest cutoff), and the blocks
    // past the last term would only add exact zeros (FP64 is scarce here:
    // their reductions had made both kernels about 0.1 ms each).
    int64_t kmax = 0;
    for (int e = 0; e < n_eps; ++e) kmax = a.kend[e] > kmax ? a.kend[e] : kmax;
    int64_t blocks = (kmax + kActThreads - 1) / kActThreads;
    blocks = blocks < 1 ? 1 : (blocks > kActBlocks ? kActBlocks : blocks);
    dd* partial = reinterpret_cast<dd*>(static_cast<uint8_t*>(workspace) + sizeof(WsHeader));
    if (any_smeared) k_action_partial<<<unsigned(blocks), kActThreads, 0, st>>>(dim, n, hist, len, a, partial);
    k_action_final<<<1, 32, 0, st>>>(dim, n, hist, len, a, partial, int(blocks), out, bracket);
    return cudaGetLastError();
}

}  // namespace cs
