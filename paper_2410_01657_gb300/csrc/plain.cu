// Plain FP32 path of libgnnmp: unfused SIMT kernels, no tensor cores, no TF32.
//
// This is the straightforward reading of the consistent NMP layer (Eq. 5a-5e)
// and its adjoint, one kernel per operation with every intermediate in
// workspace memory. It is the FP32 correctness and speed baseline the fused
// BF16 path is measured against. All reductions run in a fixed order:
// CSR segmented sums over receiver (or sender) lists, split-K partial products
// reduced in chunk order, and block-partial column sums reduced in block
// order, so two runs give bitwise equal results.

#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "plain.h"
#include "profiler.h"

namespace gnn {
namespace plain {

cudaError_t take_device_error(unsigned int* out) { return take_device_error_word(out); }

// =================================================================== kernels

struct GemmArgs {
    int64_t M, N, K;
    const float* A;
    int64_t sAm, sAk;        // A(m,k) = A[m*sAm + k*sAk]
    const float* B;
    int64_t sBk, sBn;        // B(k,n) = B[k*sBk + n*sBn]
    float* C;
    int64_t ldc;             // C[m*ldc + n]
    const float* bias;       // [N] or NULL
    int elu;                 // apply ELU to the result
    int accumulate;          // C += result
    int64_t k_chunk;         // split-K: blockIdx.z takes K range [z*k_chunk, (z+1)*k_chunk)
    int64_t c_split_stride;  // and writes C + z*c_split_stride
};

// C = op(A) op(B) (+bias, ELU) with a 64x64 block tile, 16-deep K steps and
// 4x4 outputs per thread. Operands are staged through shared memory with the
// load order chosen so that the contiguous index is the fast thread index.
__global__ void __launch_bounds__(256) k_sgemm(GemmArgs a) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * 64, n0 = (int64_t)blockIdx.y * 64;   // rows in x: up to 2^31-1 blocks
    int64_t kbeg = 0, kend = a.K;
    float* C = a.C;
    if (a.k_chunk > 0) {
        kbeg = (int64_t)blockIdx.z * a.k_chunk;
        kend = min(a.K, kbeg + a.k_chunk);
        C += (int64_t)blockIdx.z * a.c_split_stride;
    }
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int64_t k0 = kbeg; k0 < kend; k0 += 16) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int idx = threadIdx.x + i * 256;
            int mm, kk;
            if (a.sAk == 1) { kk = idx & 15; mm = idx >> 4; }
            else { mm = idx & 63; kk = idx >> 6; }
            int64_t gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < a.M && gk < kend) ? a.A[gm * a.sAm + gk * a.sAk] : 0.f;
            int nn;
            if (a.sBn == 1) { nn = idx & 63; kk = idx >> 6; }
            else { kk = idx & 15; nn = idx >> 4; }
            int64_t gn = n0 + nn;
            gk = k0 + kk;
            Bs[kk][nn] = (gn < a.N && gk < kend) ? a.B[gk * a.sBk + gn * a.sBn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t n = n0 + tx + 16 * j;
            if (n >= a.N) continue;
            float v = acc[i][j];
            if (a.bias) v += a.bias[n];
            if (a.elu) v = elu1(v);
            float* dst = C + m * a.ldc + n;
            *dst = a.accumulate ? *dst + v : v;
        }
    }
}

// out[i] (+)= sum_z part[z*n + i], z ascending.
__global__ void k_reduce_partials(const float* __restrict__ part, int64_t nsplit, int64_t n,
                                  float* __restrict__ out, int accumulate) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int64_t z = 0; z < nsplit; ++z) s += part[z * n + i];
    out[i] = accumulate ? out[i] + s : s;
}

// part[b*cols + c] = sum of X[r*ld + c] over rows r of chunk b, r ascending.
__global__ void __launch_bounds__(256) k_colsum_partial(const float* __restrict__ X, int64_t rows, int64_t ld,
                                                        int cols, int64_t chunk, float* __restrict__ part) {
    // 32 columns x 8 row lanes per pass over the chunk; the 8 partial sums of a
    // column are combined in lane order, so the result does not depend on timing.
    __shared__ float red[8][33];
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    for (int c0 = 0; c0 < cols; c0 += 32) {
        const int c = c0 + cx;
        float s = 0.f;
        if (c < cols)
            for (int64_t r = r0 + ry; r < r1; r += 8) s += X[r * ld + c];
        red[ry][cx] = s;
        __syncthreads();
        if (ry == 0 && c < cols) {
            float t = 0.f;
            for (int k = 0; k < 8; ++k) t += red[k][cx];
            part[(int64_t)blockIdx.x * cols + c] = t;
        }
        __syncthreads();
    }
}

// LayerNorm over rows of Z [rows x H] (H <= 256), one warp per row:
// out = res + gamma * (z - mean) * rstd + beta (res optional).
template <typename TR, typename TO>
__global__ void k_ln_fwd(const float* __restrict__ Z, int64_t rows, int H, const float* __restrict__ gamma,
                         const float* __restrict__ beta, float eps, const TR* __restrict__ res,
                         TO* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nwarp) {
        float v[8];
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = lane + 32 * i;
            v[i] = c < H ? Z[r * H + c] : 0.f;
            s += v[i];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float mean = s / H;
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = lane + 32 * i;
            float d = c < H ? v[i] - mean : 0.f;
            q += d * d;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        const float rstd = rsqrtf(q / H + eps);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = lane + 32 * i;
            if (c < H) {
                float y = (v[i] - mean) * rstd * gamma[c] + beta[c];
                if (res) y += to_f32(res[r * H + c]);
                out[r * H + c] = from_f32<TO>(y);
            }
        }
    }
}

// LayerNorm adjoint, one warp per row; block b owns rows [b*chunk, (b+1)*chunk)
// and writes its dgamma/dbeta partial sums (warps summed in warp order).
__global__ void __launch_bounds__(256) k_ln_bwd(const float* __restrict__ Z, const float* __restrict__ G,
                                                int64_t rows, int H, const float* __restrict__ gamma, float eps,
                                                float* __restrict__ dZ, int64_t chunk,
                                                float* __restrict__ part_g, float* __restrict__ part_b) {
    __shared__ float sg[8][256];
    __shared__ float sb[8][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float accg[8], accb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) accg[i] = accb[i] = 0.f;
    int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    for (int64_t r = r0 + w; r < r1; r += 8) {
        float v[8], g[8];
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = lane + 32 * i;
            v[i] = c < H ? Z[r * H + c] : 0.f;
            g[i] = c < H ? G[r * H + c] : 0.f;
            s += v[i];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float mean = s / H;
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = lane + 32 * i;
            float d = c < H ? v[i] - mean : 0.f;
            q += d * d;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        const float rstd = rsqrtf(q / H + eps);
        float m1 = 0.f, m2 = 0.f;
        float xh[8], dxh[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = lane + 32 * i;
            xh[i] = (v[i] - mean) * rstd;
            dxh[i] = c < H ? g[i] * gamma[c] : 0.f;
            if (c < H) {
                accg[i] += g[i] * xh[i];
                accb[i] += g[i];
            }
            m1 += dxh[i];
            m2 += dxh[i] * (c < H ? xh[i] : 0.f);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            m1 += __shfl_xor_sync(0xffffffffu, m1, o);
            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        }
        m1 /= H;
        m2 /= H;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = lane + 32 * i;
            if (c < H) dZ[r * H + c] = rstd * (dxh[i] - m1 - xh[i] * m2);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int c = lane + 32 * i;
        if (c < H) {
            sg[w][c] = accg[i];
            sb[w][c] = accb[i];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < H; c += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int k = 0; k < 8; ++k) {
            a += sg[k][c];
            b += sb[k][c];
        }
        part_g[(int64_t)blockIdx.x * H + c] = a;
        part_b[(int64_t)blockIdx.x * H + c] = b;
    }
}

// g *= ELU'(z) given h = ELU(z).
__global__ void k_elu_bwd(float* __restrict__ g, const float* __restrict__ h, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g[i] *= elu1_deriv_from_out(h[i]);
}

// X1[e] = [x[receiver], x[sender], e_in[e]] for every edge of every receiver row.
__global__ void k_gather_edge_input(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                    int64_t rows, int H, const float* __restrict__ x,
                                    const float* __restrict__ e_in, float* __restrict__ X1) {
    int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        int64_t s = col[e];
        float* dst = X1 + (int64_t)e * 3 * H;
        for (int c = lane; c < H; c += 32) {
            dst[c] = x[r * H + c];
            dst[H + c] = x[s * H + c];
            dst[2 * H + c] = e_in[(int64_t)e * H + c];
        }
    }
}

// a[r] = sum over edges e of r (ascending) of w[e] * Y[e].            (Eq. 5b)
__global__ void k_segsum(const int32_t* __restrict__ row_ptr, const float* __restrict__ w, int64_t rows, int H,
                         const float* __restrict__ Y, float* __restrict__ a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * H) return;
    int64_t r = i / H;
    int c = (int)(i - r * H);
    float s = 0.f;
    for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) s += w[e] * Y[(int64_t)e * H + c];
    a[i] = s;
}

// de_tot[e] = de_out[e] + w[e] * da[receiver(e)]    (adjoint of Eq. 5b; de_out may be NULL)
__global__ void k_agg_adjoint(const int32_t* __restrict__ row_ptr, const float* __restrict__ w, int64_t rows,
                              int H, const float* __restrict__ da, const float* __restrict__ de_out,
                              float* __restrict__ de_tot) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * H) return;
    int64_t r = i / H;
    int c = (int)(i - r * H);
    float g = da[i];
    for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        int64_t k = (int64_t)e * H + c;
        de_tot[k] = (de_out ? de_out[k] : 0.f) + w[e] * g;
    }
}

// dx[r] += sum_{e in recv(r)} dX1[e][0:H] + sum_{e in send(r)} dX1[e][H:2H]   (gather adjoint)
__global__ void k_gather_adjoint(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ t_ptr,
                                 const int32_t* __restrict__ t_eid, int64_t rows, int H,
                                 const float* __restrict__ dX1, float* __restrict__ dx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * H) return;
    int64_t r = i / H;
    int c = (int)(i - r * H);
    float s = 0.f;
    for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) s += dX1[(int64_t)e * 3 * H + c];
    float t = 0.f;
    for (int32_t k = t_ptr[r]; k < t_ptr[r + 1]; ++k) t += dX1[(int64_t)t_eid[k] * 3 * H + H + c];
    dx[i] += s + t;
}

// X2[r] = [a[r], x[r]]
__global__ void k_concat2(const float* __restrict__ a, const float* __restrict__ x, int64_t rows, int H,
                          float* __restrict__ X2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * H) return;
    int64_t r = i / H;
    int c = (int)(i - r * H);
    X2[r * 2 * H + c] = a[i];
    X2[r * 2 * H + H + c] = x[i];
}

// da[r] = dX2[r][0:H];  dx[r] = dx_out[r] + dX2[r][H:2H]
__global__ void k_split_node_grad(const float* __restrict__ dX2, const float* __restrict__ dx_out, int64_t rows,
                                  int H, float* __restrict__ da, float* __restrict__ dx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * H) return;
    int64_t r = i / H;
    int c = (int)(i - r * H);
    da[i] = dX2[r * 2 * H + c];
    dx[i] = dx_out[i] + dX2[r * 2 * H + H + c];
}

// de_in[e] = de_tot[e] + dX1[e][2H:3H]      (residual + edge-state part of the input)
__global__ void k_edge_grad_out(const float* __restrict__ de_tot, const float* __restrict__ dX1, int64_t E, int H,
                                float* __restrict__ de_in) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E * H) return;
    int64_t e = i / H;
    int c = (int)(i - e * H);
    de_in[i] = de_tot[i] + dX1[e * 3 * H + 2 * H + c];
}

// Eq. 5c-5d on one device: each shared id's copies are summed in list order
// (increasing sub-graph) and the sum written back to every copy.
__global__ void k_halo(const int32_t* __restrict__ halo_ptr, const int32_t* __restrict__ halo_rows,
                       int64_t n_shared, int H, float* __restrict__ rows) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_shared * H) return;
    int64_t s = i / H;
    int c = (int)(i - s * H);
    int32_t k0 = halo_ptr[s], k1 = halo_ptr[s + 1];
    float v = 0.f;
    for (int32_t k = k0; k < k1; ++k) v += rows[(int64_t)halo_rows[k] * H + c];
    for (int32_t k = k0; k < k1; ++k) rows[(int64_t)halo_rows[k] * H + c] = v;
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ in, float* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __bfloat162float(in[i]);
}

__global__ void k_f32_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// Consistent loss, Eq. 8: block partials of sum w_i (y-t)^2 and of sum w_i.
__global__ void __launch_bounds__(256) k_loss_partial(const float* __restrict__ y, const float* __restrict__ t,
                                                      const float* __restrict__ w, int64_t rows, int F,
                                                      int64_t chunk, float* __restrict__ part) {
    __shared__ float s1[256], s2[256];
    int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    float a = 0.f, b = 0.f;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        float q = 0.f;
        for (int f = 0; f < F; ++f) {
            float d = y[r * F + f] - t[r * F + f];
            q += d * d;
        }
        a += w[r] * q;
        b += w[r];
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

// loss = S / (N_eff F); stats[0] = loss, stats[1] = N_eff.
__global__ void k_loss_final(const float* __restrict__ part, int64_t nblk, int F, float* __restrict__ loss,
                             float* __restrict__ stats) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double S = 0.0, Ne = 0.0;
    for (int64_t b = 0; b < nblk; ++b) {
        S += part[2 * b];
        Ne += part[2 * b + 1];
    }
    float L = (float)(S / (Ne * F));
    *loss = L;
    stats[0] = L;
    stats[1] = (float)Ne;
}

__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ w,
                            int64_t rows, int F, const float* __restrict__ stats, float* __restrict__ dy) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * F) return;
    int64_t r = i / F;
    dy[i] = 2.f * (y[i] - t[i]) * w[r] / (stats[1] * F);
}

// =================================================================== host helpers

static inline unsigned grid1(int64_t n, int threads = 256) { return (unsigned)((n + threads - 1) / threads); }

static int gemm(const GemmArgs& a, int64_t nsplit, cudaStream_t s) {
    if (a.M == 0 || a.N == 0) return GNN_OK;
    const int64_t mb = (a.M + 63) / 64;
    GNN_REQUIRE(mb <= 0x7fffffff, GNN_ESHAPE, "sgemm: too many rows");
    dim3 grid((unsigned)mb, (unsigned)((a.N + 63) / 64), (unsigned)std::max<int64_t>(1, nsplit));
    GNN_REQUIRE(grid.y <= 65535u && grid.z <= 65535u, GNN_ESHAPE, "sgemm: grid too large");
    {
        ProfScope _ps(s, "k_sgemm");
        k_sgemm<<<grid, 256, 0, s>>>(a);
    }
    GNN_LAUNCH_CHECK("k_sgemm");
    return GNN_OK;
}

// Y[rows x N] = X[rows x K] W^T + b (+ELU)
static int linear_fwd(int64_t rows, int64_t K, int64_t N, const float* X, int64_t ldx, const float* W,
                      const float* b, float* Y, int elu, cudaStream_t s) {
    GemmArgs a{};
    a.M = rows; a.N = N; a.K = K;
    a.A = X; a.sAm = ldx; a.sAk = 1;
    a.B = W; a.sBk = 1; a.sBn = K;
    a.C = Y; a.ldc = N; a.bias = b; a.elu = elu;
    return gemm(a, 1, s);
}

// dX[rows x K] (+)= G[rows x N] W[N x K]
static int linear_bwd_data(int64_t rows, int64_t K, int64_t N, const float* G, const float* W, float* dX,
                           int64_t lddx, cudaStream_t s) {
    GemmArgs a{};
    a.M = rows; a.N = K; a.K = N;
    a.A = G; a.sAm = N; a.sAk = 1;
    a.B = W; a.sBk = K; a.sBn = 1;
    a.C = dX; a.ldc = lddx;
    return gemm(a, 1, s);
}

int64_t chunk_rows(int64_t rows) { return std::max<int64_t>(4096, (rows + 511) / 512); }
int64_t n_chunks(int64_t rows) { return rows == 0 ? 0 : (rows + chunk_rows(rows) - 1) / chunk_rows(rows); }

// dW[N x K] += G^T X over all rows (split-K over row chunks, reduced in chunk order);
// db[N] += column sums of G.
static int linear_bwd_weight(int64_t rows, int64_t K, int64_t N, const float* G, const float* X, int64_t ldx,
                             float* dW, float* db, float* part, cudaStream_t s) {
    if (rows == 0) return GNN_OK;
    const int64_t ch = chunk_rows(rows), nz = n_chunks(rows);
    GemmArgs a{};
    a.M = N; a.N = K; a.K = rows;
    a.A = G; a.sAm = 1; a.sAk = N;
    a.B = X; a.sBk = ldx; a.sBn = 1;
    a.C = part; a.ldc = K;
    a.k_chunk = ch; a.c_split_stride = N * K;
    int rc = gemm(a, nz, s);
    if (rc) return rc;
    {
        ProfScope _ps(s, "k_reduce_partials");
        k_reduce_partials<<<grid1(N * K), 256, 0, s>>>(part, nz, N * K, dW, 1);
    }
    GNN_LAUNCH_CHECK("k_reduce_partials");
    if (db) {
        {
            ProfScope _ps(s, "k_colsum_partial");
            k_colsum_partial<<<(unsigned)nz, 256, 0, s>>>(G, rows, N, (int)N, ch, part);
        }
        GNN_LAUNCH_CHECK("k_colsum_partial");
        {
            ProfScope _ps(s, "k_reduce_partials");
            k_reduce_partials<<<grid1(N), 256, 0, s>>>(part, nz, N, db, 1);
        }
        GNN_LAUNCH_CHECK("k_reduce_partials");
    }
    return GNN_OK;
}

size_t partial_floats(const gnn_mlp& P, int64_t rows) {
    int64_t mx = 0;
    for (int k = 0; k < P.n_lin; ++k) mx = std::max<int64_t>(mx, (int64_t)P.dims[k] * P.dims[k + 1]);
    mx = std::max<int64_t>(mx, 2 * P.dims[P.n_lin]);
    return (size_t)(n_chunks(rows) * mx + 64);
}

int max_width(const gnn_mlp& P) {
    int m = 0;
    for (int k = 0; k <= P.n_lin; ++k) m = std::max(m, P.dims[k]);
    return m;
}

// Forward of the Linear/ELU chain. hbuf[k] (k = 1..n_lin-1) receives the
// input of Linear k (an ELU output); zlast receives the last Linear's output.
int chain_fwd(const gnn_mlp& P, int64_t rows, const float* X, int64_t ldx, float* const* hbuf, float* zlast,
              cudaStream_t s) {
    const float* in = X;
    int64_t ld = ldx;
    for (int k = 0; k < P.n_lin; ++k) {
        const bool last = (k == P.n_lin - 1);
        float* out = last ? zlast : hbuf[k + 1];
        int rc = linear_fwd(rows, P.dims[k], P.dims[k + 1], in, ld, P.W[k], P.b[k], out, last ? 0 : 1, s);
        if (rc) return rc;
        in = out;
        ld = P.dims[k + 1];
    }
    return GNN_OK;
}

template <typename TR, typename TO>
static int ln_fwd(const float* Z, int64_t rows, int H, const gnn_mlp& P, float eps, const TR* res, TO* out,
                  cudaStream_t s) {
    if (rows == 0) return GNN_OK;
    unsigned blocks = (unsigned)std::min<int64_t>((rows + 7) / 8, 152 * 16);
    {
        ProfScope _ps(s, "k_ln_fwd");
        k_ln_fwd<TR, TO><<<blocks, 256, 0, s>>>(Z, rows, H, P.gamma, P.beta, eps, res, out);
    }
    GNN_LAUNCH_CHECK("k_ln_fwd");
    return GNN_OK;
}

// Output of an MLP from its last pre-activation: LayerNorm (+ residual) or a copy.
int mlp_output(const gnn_mlp& P, int64_t rows, const float* zlast, float eps, const float* res_f32,
               const __nv_bfloat16* res_bf16, void* out, int out_bf16, cudaStream_t s) {
    const int H = P.dims[P.n_lin];
    if (P.gamma) {
        if (out_bf16) {
            if (res_bf16) return ln_fwd<__nv_bfloat16, __nv_bfloat16>(zlast, rows, H, P, eps, res_bf16, (__nv_bfloat16*)out, s);
            return ln_fwd<float, __nv_bfloat16>(zlast, rows, H, P, eps, res_f32, (__nv_bfloat16*)out, s);
        }
        if (res_bf16) return ln_fwd<__nv_bfloat16, float>(zlast, rows, H, P, eps, res_bf16, (float*)out, s);
        return ln_fwd<float, float>(zlast, rows, H, P, eps, res_f32, (float*)out, s);
    }
    GNN_REQUIRE(!res_f32 && !res_bf16, GNN_EINVAL, "mlp_output: residual without LayerNorm is not supported");
    if (rows == 0) return GNN_OK;
    if (out_bf16) {
        {
            ProfScope _ps(s, "k_f32_to_bf16");
            k_f32_to_bf16<<<grid1(rows * H), 256, 0, s>>>(zlast, (__nv_bfloat16*)out, rows * H);
        }
        GNN_LAUNCH_CHECK("k_f32_to_bf16");
    } else if (out != zlast) {
        GNN_CUDA_CHECK(cudaMemcpyAsync(out, zlast, sizeof(float) * rows * H, cudaMemcpyDeviceToDevice, s), "copy");
    }
    return GNN_OK;
}

// Adjoint of chain_fwd + mlp_output. dY: [rows x out] gradient of the MLP
// output (before any residual). X/hbuf/zlast: the recomputed forward.
// g0, g1: [rows x max_width] scratch. dX: [rows x dims[0]] written, or NULL.
int mlp_bwd(const gnn_mlp& P, const gnn_mlp& dP, int64_t rows, const float* X, int64_t ldx, float* const* hbuf,
            const float* zlast, const float* dY, float* dX, float* g0, float* g1, float* part, float eps,
            cudaStream_t s) {
    const int n = P.n_lin;
    const int H = P.dims[n];
    float* g = g0;
    float* gn = g1;
    if (P.gamma) {
        const int64_t ch = chunk_rows(rows), nz = n_chunks(rows);
        if (rows) {
            {
                ProfScope _ps(s, "k_ln_bwd");
                k_ln_bwd<<<(unsigned)nz, 256, 0, s>>>(zlast, dY, rows, H, P.gamma, eps, g, ch, part, part + nz * H);
            }
            GNN_LAUNCH_CHECK("k_ln_bwd");
            {
                ProfScope _ps(s, "k_reduce_partials");
                k_reduce_partials<<<grid1(H), 256, 0, s>>>(part, nz, H, dP.gamma, 1);
            }
            GNN_LAUNCH_CHECK("k_reduce_partials");
            {
                ProfScope _ps(s, "k_reduce_partials");
                k_reduce_partials<<<grid1(H), 256, 0, s>>>(part + nz * H, nz, H, dP.beta, 1);
            }
            GNN_LAUNCH_CHECK("k_reduce_partials");
        }
    } else if (rows) {
        GNN_CUDA_CHECK(cudaMemcpyAsync(g, dY, sizeof(float) * rows * H, cudaMemcpyDeviceToDevice, s), "copy");
    }
    for (int k = n - 1; k >= 0; --k) {
        const float* in = (k == 0) ? X : hbuf[k];
        const int64_t ld = (k == 0) ? ldx : P.dims[k];
        int rc = linear_bwd_weight(rows, P.dims[k], P.dims[k + 1], g, in, ld, dP.W[k], dP.b[k], part, s);
        if (rc) return rc;
        if (k > 0) {
            rc = linear_bwd_data(rows, P.dims[k], P.dims[k + 1], g, P.W[k], gn, P.dims[k], s);
            if (rc) return rc;
            if (rows) {
                {
                    ProfScope _ps(s, "k_elu_bwd");
                    k_elu_bwd<<<grid1(rows * P.dims[k]), 256, 0, s>>>(gn, hbuf[k], rows * P.dims[k]);
                }
                GNN_LAUNCH_CHECK("k_elu_bwd");
            }
            std::swap(g, gn);
        } else if (dX) {
            rc = linear_bwd_data(rows, P.dims[0], P.dims[1], g, P.W[0], dX, P.dims[0], s);
            if (rc) return rc;
        }
    }
    return GNN_OK;
}

// Workspace carving: a bump allocator over the caller's buffer (or a size
// count when base is NULL), 256-byte aligned pieces.
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* b) : base((char*)b) {}
    template <class T>
    T* take(int64_t n) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += sizeof(T) * (size_t)std::max<int64_t>(n, 0);
        return p;
    }
};

// ------------------------------------------------------------------ MP layer, plain FP32

struct LayerFwdBufs {
    float* X1;
    float* hE[GNN_MAX_LIN];
    float* zE;
    float* e_new;
    float* a;
    float* X2;
    float* hN[GNN_MAX_LIN];
    float* zN;
};

// store_acts: keep every activation (backward recompute); otherwise reuse two buffers.
static void carve_layer(Carve& c, int64_t NR, int64_t E, int H, int n_lin, bool store_acts, bool need_e_new,
                        bool need_a, LayerFwdBufs& b) {
    b.X1 = c.take<float>(E * 3 * H);
    float* pingpong[2] = {nullptr, nullptr};
    if (!store_acts) {
        int64_t m = std::max(E, NR);
        pingpong[0] = c.take<float>(m * H);
        pingpong[1] = c.take<float>(m * H);
    }
    for (int k = 1; k < n_lin; ++k) b.hE[k] = store_acts ? c.take<float>(E * H) : pingpong[k & 1];
    b.zE = c.take<float>(E * H);
    b.e_new = need_e_new ? c.take<float>(E * H) : nullptr;
    b.a = need_a ? c.take<float>(NR * H) : nullptr;
    b.X2 = c.take<float>(NR * 2 * H);
    for (int k = 1; k < n_lin; ++k) b.hN[k] = store_acts ? c.take<float>(NR * H) : pingpong[k & 1];
    b.zN = c.take<float>(NR * H);
}

static int layer_forward_core(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                              const float* x_in, const float* e_in, float* e_new, float* a, float* x_out,
                              LayerFwdBufs& b, bool skip_agg, cudaStream_t s) {
    const int H = cfg.hidden;
    const int64_t NR = G.n_rows, E = G.n_edges;
    int rc;
    if (NR && E) {
        {
            ProfScope _ps(s, "k_gather_edge_input");
            k_gather_edge_input<<<grid1(NR, 8), 256, 0, s>>>(G.row_ptr, G.col, NR, H, x_in, e_in, b.X1);
        }
        GNN_LAUNCH_CHECK("k_gather_edge_input");
    }
    if ((rc = chain_fwd(W.edge, E, b.X1, 3 * H, b.hE, b.zE, s))) return rc;
    if (!skip_agg) {
        if ((rc = mlp_output(W.edge, E, b.zE, cfg.ln_eps, e_in, nullptr, e_new, 0, s))) return rc;   // Eq. 5a
        if (NR) {
            {
                ProfScope _ps(s, "k_segsum");
                k_segsum<<<grid1(NR * H), 256, 0, s>>>(G.row_ptr, G.edge_w, NR, H, e_new, a);           // Eq. 5b
            GNN_LAUNCH_CHECK("k_segsum");
            }
        }
        if (cfg.halo_mode == GNN_HALO_SYNC && G.n_shared) {                                      // Eq. 5c-5d
            {
                ProfScope _ps(s, "k_halo");
                k_halo<<<grid1(G.n_shared * H), 256, 0, s>>>(G.halo_ptr, G.halo_rows, G.n_shared, H, a);
            }
            GNN_LAUNCH_CHECK("k_halo");
        }
    }
    if (NR) {
        {
            ProfScope _ps(s, "k_concat2");
            k_concat2<<<grid1(NR * H), 256, 0, s>>>(a, x_in, NR, H, b.X2);
        }
        GNN_LAUNCH_CHECK("k_concat2");
    }
    if ((rc = chain_fwd(W.node, NR, b.X2, 2 * H, b.hN, b.zN, s))) return rc;
    if (x_out) {
        if ((rc = mlp_output(W.node, NR, b.zN, cfg.ln_eps, x_in, nullptr, x_out, 0, s))) return rc;   // Eq. 5e
    }
    return GNN_OK;
}

size_t mp_forward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W) {
    Carve c(nullptr);
    LayerFwdBufs b;
    carve_layer(c, G.n_rows, G.n_edges, cfg.hidden, std::max(W.edge.n_lin, W.node.n_lin), false, true, true, b);
    return c.off + 256;
}

int mp_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
               const float* e_in, float* x_out, float* e_out, float* a_star_out, void* ws, size_t ws_bytes,
               cudaStream_t s) {
    GNN_REQUIRE(ws_bytes >= mp_forward_ws(G, cfg, W), GNN_ENOMEM, "gnn_mp_forward: workspace too small");
    Carve c(ws);
    LayerFwdBufs b;
    carve_layer(c, G.n_rows, G.n_edges, cfg.hidden, std::max(W.edge.n_lin, W.node.n_lin), false, true, true, b);
    float* e_new = e_out ? e_out : b.e_new;
    float* a = a_star_out ? a_star_out : b.a;
    return layer_forward_core(G, cfg, W, x_in, e_in, e_new, a, x_out, b, false, s);
}

struct LayerBwdBufs {
    float* g0;
    float* g1;
    float* dX1;
    float* de_tot;
    float* dX2;
    float* da;
    float* part;
    float* dY;
};

static void carve_bwd(Carve& c, const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                      LayerBwdBufs& d) {
    const int H = cfg.hidden;
    const int64_t NR = G.n_rows, E = G.n_edges, m = std::max(NR, E);
    const int wmax = std::max(max_width(W.edge), max_width(W.node));
    d.g0 = c.take<float>(m * wmax);
    d.g1 = c.take<float>(m * wmax);
    d.dX1 = c.take<float>(E * 3 * H);
    d.de_tot = c.take<float>(E * H);
    d.dX2 = c.take<float>(NR * 2 * H);
    d.da = c.take<float>(NR * H);
    d.part = c.take<float>((int64_t)std::max(partial_floats(W.edge, E), partial_floats(W.node, NR)));
    d.dY = c.take<float>(0);
}

size_t mp_backward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W) {
    Carve c(nullptr);
    LayerFwdBufs b;
    LayerBwdBufs d;
    carve_layer(c, G.n_rows, G.n_edges, cfg.hidden, std::max(W.edge.n_lin, W.node.n_lin), true, true, true, b);
    carve_bwd(c, G, cfg, W, d);
    return c.off + 256;
}

int mp_backward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                const float* e_in, const float* a_star, const float* dx_out, const float* de_out, float* dx_in,
                float* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes, cudaStream_t s) {
    GNN_REQUIRE(ws_bytes >= mp_backward_ws(G, cfg, W), GNN_ENOMEM, "gnn_mp_backward: workspace too small");
    const int H = cfg.hidden;
    const int64_t NR = G.n_rows, E = G.n_edges;
    Carve c(ws);
    LayerFwdBufs b;
    LayerBwdBufs d;
    carve_layer(c, NR, E, H, std::max(W.edge.n_lin, W.node.n_lin), true, true, true, b);
    carve_bwd(c, G, cfg, W, d);
    int rc;
    // recompute the forward activations of this layer
    float* a = b.a;
    if (a_star) {
        if (NR) GNN_CUDA_CHECK(cudaMemcpyAsync(a, a_star, sizeof(float) * NR * H, cudaMemcpyDeviceToDevice, s), "copy");
    }
    if ((rc = layer_forward_core(G, cfg, W, x_in, e_in, b.e_new, a, nullptr, b, a_star != nullptr, s))) return rc;

    // node update adjoint (Eq. 5e)
    if ((rc = mlp_bwd(W.node, dW.node, NR, b.X2, 2 * H, b.hN, b.zN, dx_out, d.dX2, d.g0, d.g1, d.part, cfg.ln_eps, s)))
        return rc;
    if (NR) {
        {
            ProfScope _ps(s, "k_split_node_grad");
            k_split_node_grad<<<grid1(NR * H), 256, 0, s>>>(d.dX2, dx_out, NR, H, d.da, dx_in);
        }
        GNN_LAUNCH_CHECK("k_split_node_grad");
    }
    // halo swap + sync adjoint (Eq. 5c-5d): the same symmetric copy-sum
    if (cfg.halo_mode == GNN_HALO_SYNC && G.n_shared) {
        {
            ProfScope _ps(s, "k_halo");
            k_halo<<<grid1(G.n_shared * H), 256, 0, s>>>(G.halo_ptr, G.halo_rows, G.n_shared, H, d.da);
        }
        GNN_LAUNCH_CHECK("k_halo");
    }
    // aggregation adjoint (Eq. 5b) + upstream edge gradient
    if (NR) {
        {
            ProfScope _ps(s, "k_agg_adjoint");
            k_agg_adjoint<<<grid1(NR * H), 256, 0, s>>>(G.row_ptr, G.edge_w, NR, H, d.da, de_out, d.de_tot);
        }
        GNN_LAUNCH_CHECK("k_agg_adjoint");
    }
    // edge update adjoint (Eq. 5a)
    if ((rc = mlp_bwd(W.edge, dW.edge, E, b.X1, 3 * H, b.hE, b.zE, d.de_tot, d.dX1, d.g0, d.g1, d.part, cfg.ln_eps, s)))
        return rc;
    if (E) {
        {
            ProfScope _ps(s, "k_edge_grad_out");
            k_edge_grad_out<<<grid1(E * H), 256, 0, s>>>(d.de_tot, d.dX1, E, H, de_in);
        }
        GNN_LAUNCH_CHECK("k_edge_grad_out");
    }
    if (NR) {
        {
            ProfScope _ps(s, "k_gather_adjoint");
            k_gather_adjoint<<<grid1(NR * H), 256, 0, s>>>(G.row_ptr, G.t_ptr, G.t_eid, NR, H, d.dX1, dx_in);
        }
        GNN_LAUNCH_CHECK("k_gather_adjoint");
    }
    return GNN_OK;
}

int halo(const gnn_graph_dev& G, float* rows, int width, cudaStream_t s) {
    if (G.n_shared == 0 || width == 0) return GNN_OK;
    {
        ProfScope _ps(s, "k_halo");
        k_halo<<<grid1(G.n_shared * width), 256, 0, s>>>(G.halo_ptr, G.halo_rows, G.n_shared, width, rows);
    }
    GNN_LAUNCH_CHECK("k_halo");
    return GNN_OK;
}

// ------------------------------------------------------------------ row-wise MLP (encoders/decoder)

static void carve_mlp(Carve& c, const gnn_mlp& P, int64_t rows, bool bwd, float** h, float** z, float** g0,
                      float** g1, float** part, float** dYf) {
    const int wmax = max_width(P);
    for (int k = 1; k < P.n_lin; ++k) h[k] = c.take<float>(rows * P.dims[k]);
    *z = c.take<float>(rows * P.dims[P.n_lin]);
    if (bwd) {
        *g0 = c.take<float>(rows * wmax);
        *g1 = c.take<float>(rows * wmax);
        *part = c.take<float>((int64_t)partial_floats(P, rows));
        *dYf = c.take<float>(rows * P.dims[P.n_lin]);
    }
}

// The row MLP runs over blocks of at most kMlpRowBlock rows: its workspace
// (every activation of a block, FP32) is sized for one block, so an encoder
// over tens of millions of edge rows needs a bounded workspace. The weight
// gradients accumulate block after block, in row order.
constexpr int64_t kMlpRowBlock = (int64_t)1 << 22;

size_t mlp_ws(const gnn_mlp& P, int64_t rows, bool bwd) {
    Carve c(nullptr);
    float *h[GNN_MAX_LIN], *z, *g0, *g1, *part, *dy;
    carve_mlp(c, P, std::min(rows, kMlpRowBlock), bwd, h, &z, &g0, &g1, &part, &dy);
    return c.off + 256;
}

int mlp_forward(const gnn_mlp& P, int64_t rows, const float* X, void* Y, int y_bf16, float eps, void* ws,
                size_t ws_bytes, cudaStream_t s) {
    GNN_REQUIRE(ws_bytes >= mlp_ws(P, rows, false), GNN_ENOMEM, "gnn_mlp_forward: workspace too small");
    const int K0 = P.dims[0], NO = P.dims[P.n_lin];
    for (int64_t r0 = 0; r0 < rows; r0 += kMlpRowBlock) {
        const int64_t n = std::min(kMlpRowBlock, rows - r0);
        Carve c(ws);
        float *h[GNN_MAX_LIN], *z, *g0, *g1, *part, *dy;
        carve_mlp(c, P, n, false, h, &z, &g0, &g1, &part, &dy);
        int rc = chain_fwd(P, n, X + r0 * K0, K0, h, z, s);
        if (rc) return rc;
        void* Yb = (char*)Y + (size_t)(r0 * NO) * (y_bf16 ? 2 : 4);
        if ((rc = mlp_output(P, n, z, eps, nullptr, nullptr, Yb, y_bf16, s))) return rc;
    }
    return GNN_OK;
}

int mlp_backward(const gnn_mlp& P, int64_t rows, const float* X, const void* dY, int dy_bf16, float* dX,
                 const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s) {
    GNN_REQUIRE(ws_bytes >= mlp_ws(P, rows, true), GNN_ENOMEM, "gnn_mlp_backward: workspace too small");
    const int K0 = P.dims[0], NO = P.dims[P.n_lin];
    for (int64_t r0 = 0; r0 < rows; r0 += kMlpRowBlock) {
        const int64_t n = std::min(kMlpRowBlock, rows - r0);
        Carve c(ws);
        float *h[GNN_MAX_LIN], *z, *g0, *g1, *part, *dyf;
        carve_mlp(c, P, n, true, h, &z, &g0, &g1, &part, &dyf);
        const float* Xb = X + r0 * K0;
        int rc = chain_fwd(P, n, Xb, K0, h, z, s);
        if (rc) return rc;
        const float* dy = (const float*)dY + r0 * NO;
        if (dy_bf16) {
            {
                ProfScope _ps(s, "k_bf16_to_f32");
                k_bf16_to_f32<<<grid1(n * NO), 256, 0, s>>>((const __nv_bfloat16*)dY + r0 * NO, dyf, n * NO);
            }
            GNN_LAUNCH_CHECK("k_bf16_to_f32");
            dy = dyf;
        }
        if ((rc = mlp_bwd(P, dP, n, Xb, K0, h, z, dy, dX ? dX + r0 * K0 : nullptr, g0, g1, part, eps, s)))
            return rc;
    }
    return GNN_OK;
}

int consistent_loss(const gnn_graph_dev& G, const float* y, const float* t, int F, float* loss, float* dy,
                    void* ws, size_t ws_bytes, cudaStream_t s) {
    const int64_t rows = G.n_rows;
    const int64_t chunk = std::max<int64_t>(4096, (rows + 1023) / 1024);
    const int64_t nblk = std::max<int64_t>(1, (rows + chunk - 1) / chunk);
    GNN_REQUIRE(ws_bytes >= (size_t)(2 * nblk + 2) * sizeof(float) + 256, GNN_ENOMEM,
                "gnn_consistent_loss: workspace too small");
    float* part = (float*)ws;
    float* stats = part + 2 * nblk;
    {
        ProfScope _ps(s, "k_loss_partial");
        k_loss_partial<<<(unsigned)nblk, 256, 0, s>>>(y, t, G.node_w, rows, F, chunk, part);
    }
    GNN_LAUNCH_CHECK("k_loss_partial");
    {
        ProfScope _ps(s, "k_loss_final");
        k_loss_final<<<1, 32, 0, s>>>(part, nblk, F, loss, stats);
    }
    GNN_LAUNCH_CHECK("k_loss_final");
    if (dy && rows) {
        {
            ProfScope _ps(s, "k_loss_grad");
            k_loss_grad<<<grid1(rows * F), 256, 0, s>>>(y, t, G.node_w, rows, F, stats, dy);
        }
        GNN_LAUNCH_CHECK("k_loss_grad");
    }
    return GNN_OK;
}

}  // namespace plain
}  // namespace gnn
