// Quality metrics of a drawing X of the graph (Section 4.1.3).
//
// Neighbourhood preservation, radius r: for a vertex v, N_G(v, r) is the set
// of other vertices within r hops, and N_D(v, r) the |N_G(v, r)| other
// vertices closest to v in the drawing; the metric is the sum over v of
// |N_G cap N_D| / |N_G cup N_D|. np_kernel takes one CTA per vertex:
//   1. the r-hop ball as a bitmap in shared memory, level by level (a
//      frontier bitmap expanded by one warp per 32-vertex word);
//   2. the |N_G|-th smallest key (squared distance, id) over the other
//      vertices, by radix selection: four passes of 8-bit digits over the
//      FP32 squared distance's bits (monotone for non-negative floats), then,
//      if the threshold distance is shared by more vertices than are still
//      needed, passes over the ids of those ties;
//   3. the vertices of the ball whose key is at most that threshold.
// The squared distance is summed coordinate by coordinate with explicitly
// rounded single-precision steps (no fused multiply-add), so the order of
// the drawing's distances, and thus every count, is that of the IEEE single
// arithmetic the FP32 definition states.
//
// Stress: 1/(n^2 - n) sum over ordered pairs i != j of
// ((d_ij - |X_i - X_j|) / d_ij)^2 with d_ij the hop distance, a pair with no
// path adding 1. stress_rows_kernel reads the all-pairs hop-distance rows
// (from the bit-parallel BFS of msbfs.cu), one warp per row. A term cancels
// in d_ij - |X_i - X_j| when the drawing is good, so that difference is taken
// in FP64: the squared norm from FP64 coordinate differences (exact for
// float inputs), its square root in FP32 refined by one Newton step on the
// FP64 residual; the division by d_ij and the square are FP32 (about 3e-7
// relative per term); each row's sum is FP64.
#include "gumap_internal.cuh"

#include <climits>

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kNpThreads = 256;
constexpr int kNpWarps = kNpThreads / 32;

__device__ __forceinline__ float sqdist32(const float* __restrict__ X, int dim, int u, int v) {
    float acc = 0.0f;
    for (int c = 0; c < dim; ++c) {
        const float dx = __fsub_rn(__ldg(X + (size_t)u * dim + c), __ldg(X + (size_t)v * dim + c));
        acc = __fadd_rn(acc, __fmul_rn(dx, dx));
    }
    return acc;
}

__device__ __forceinline__ bool bit_of(const uint32_t* b, int u) { return (b[u >> 5] >> (u & 31)) & 1u; }

// Block-wide sum of one value per thread (all threads call it).
__device__ __forceinline__ unsigned block_sum(unsigned x, unsigned* s_red) {
    x = __reduce_add_sync(kFull, x);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned t = 0;
    for (int w = 0; w < kNpWarps; ++w) t += s_red[w];
    return t;
}

// One selection pass: the 256-bin histogram of the digit at `shift` of the
// keys key(u) of the candidates (u != v whose key's bits above the digit
// equal `prefix`, i.e. agree under `mask`), then the bin in which the
// target-th candidate (1-based) falls. Returns the digit; *before receives
// the candidates in lower bins, *in_bin those in the chosen bin.
template <typename KeyFn>
__device__ int select_digit(int n, int v, KeyFn key, unsigned prefix, unsigned mask, int shift, unsigned target,
                            unsigned (*hist)[256], unsigned* s_sel, unsigned* before, unsigned* in_bin) {
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kNpWarps * 256; i += kNpThreads) (&hist[0][0])[i] = 0u;
    __syncthreads();
    for (int u = threadIdx.x; u < n; u += kNpThreads) {
        if (u == v) continue;
        const unsigned kb = key(u);
        if ((kb & mask) == prefix) atomicAdd(&hist[warp][(kb >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    // bin totals and their prefix: thread b owns bin b
    unsigned cnt = 0;
    for (int w = 0; w < kNpWarps; ++w) cnt += hist[w][threadIdx.x];
    unsigned inc = cnt;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();  // hist[0] is reused for the per-warp totals below
    if (lane == 31) hist[0][warp] = inc;
    __syncthreads();
    unsigned base = 0;
    for (int w = 0; w < warp; ++w) base += hist[0][w];
    const unsigned lo = base + inc - cnt, hi = base + inc;
    if (cnt > 0 && lo < target && target <= hi) {
        s_sel[0] = threadIdx.x;
        s_sel[1] = lo;
        s_sel[2] = cnt;
    }
    __syncthreads();
    const int d = (int)s_sel[0];
    *before = s_sel[1];
    *in_bin = s_sel[2];
    __syncthreads();  // s_sel and hist are rewritten by the next pass
    return d;
}

// One CTA per vertex (grid-stride). Shared memory: ball, frontier and next
// bitmaps of (n + 31) / 32 words each, and the per-warp histograms.
__global__ void __launch_bounds__(kNpThreads) np_kernel(const int32_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col, int n,
                                                        const float* __restrict__ X, int dim, int r,
                                                        int32_t* __restrict__ out_c, int32_t* __restrict__ out_inter,
                                                        double* __restrict__ out_term) {
    extern __shared__ uint32_t np_smem[];
    __shared__ unsigned hist[kNpWarps][256];
    __shared__ unsigned s_sel[4];
    __shared__ unsigned s_red[kNpWarps];
    const int words = (n + 31) >> 5;
    uint32_t* ball = np_smem;
    uint32_t* front = ball + words;
    uint32_t* next = front + words;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = blockIdx.x; v < n; v += gridDim.x) {
        // 1. the ball: v and every vertex within r hops (v removed afterwards)
        for (int i = threadIdx.x; i < words; i += kNpThreads) {
            ball[i] = 0u;
            front[i] = 0u;
            next[i] = 0u;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            ball[v >> 5] |= 1u << (v & 31);
            front[v >> 5] |= 1u << (v & 31);
        }
        __syncthreads();
        for (int d = 1; d <= r; ++d) {
            unsigned any = 0;
            for (int wd = warp; wd < words; wd += kNpWarps) {
                uint32_t fw = front[wd];
                while (fw) {
                    const int u = wd * 32 + __ffs(fw) - 1;
                    fw &= fw - 1u;
                    const int e1 = __ldg(row_ptr + u + 1);
                    for (int e = __ldg(row_ptr + u) + lane; e < e1; e += 32) {
                        const int x = __ldg(col + e);
                        const uint32_t bit = 1u << (x & 31);
                        if (!(atomicOr(&ball[x >> 5], bit) & bit)) {
                            atomicOr(&next[x >> 5], bit);
                            any = 1;
                        }
                    }
                }
            }
            const bool more = __syncthreads_or(any) != 0;
            for (int i = threadIdx.x; i < words; i += kNpThreads) {
                front[i] = next[i];
                next[i] = 0u;
            }
            __syncthreads();
            if (!more) break;
        }
        if (threadIdx.x == 0) ball[v >> 5] &= ~(1u << (v & 31));
        __syncthreads();
        unsigned pc = 0;
        for (int i = threadIdx.x; i < words; i += kNpThreads) pc += __popc(ball[i]);
        const unsigned c = block_sum(pc, s_red);

        // 2. the c-th smallest (squared distance, id) among the other vertices
        unsigned inter = 0;
        if (c > 0) {
            auto dkey = [&](int u) { return __float_as_uint(sqdist32(X, dim, u, v)); };
            unsigned target = c, prefix = 0, mask = 0;
            unsigned before = 0, in_bin = 0;
            for (int shift = 24; shift >= 0; shift -= 8) {
                const int dg = select_digit(n, v, dkey, prefix, mask, shift, target, hist, s_sel, &before, &in_bin);
                prefix |= (unsigned)dg << shift;
                mask |= 0xFFu << shift;
                target -= before;
            }
            const unsigned T = prefix;  // the threshold distance's bits; target ties of it are taken
            unsigned idT = 0xFFFFFFFFu;  // every tie taken, unless fewer are needed
            if (target < in_bin) {
                // the target-th smallest id among the vertices at distance T
                auto ikey = [&](int u) { return dkey(u) == T ? (unsigned)u : 0xFFFFFFFFu; };
                unsigned ip = 0, im = 0;
                for (int shift = 24; shift >= 0; shift -= 8) {
                    const int dg = select_digit(n, v, ikey, ip, im, shift, target, hist, s_sel, &before, &in_bin);
                    ip |= (unsigned)dg << shift;
                    im |= 0xFFu << shift;
                    target -= before;
                }
                idT = ip;
            }
            // 3. the ball's vertices at or below the threshold key
            unsigned mine = 0;
            for (int u = threadIdx.x; u < n; u += kNpThreads) {
                if (!bit_of(ball, u)) continue;
                const unsigned kb = dkey(u);
                if (kb < T || (kb == T && (unsigned)u <= idT)) ++mine;
            }
            inter = block_sum(mine, s_red);
        }
        if (threadIdx.x == 0) {
            if (out_c) out_c[v] = (int32_t)c;
            if (out_inter) out_inter[v] = (int32_t)inter;
            out_term[v] = c == 0 ? 1.0 : (double)inter / (double)(2 * c - inter);
        }
        __syncthreads();
    }
}

// One warp per all-pairs row (rows are the sources src_lo + row): the row's
// sum of stress terms in FP64.
__global__ void __launch_bounds__(256) stress_rows_kernel(const uint16_t* __restrict__ D, long long ld, int rows,
                                                          int src_lo, int n, const float* __restrict__ X, int dim,
                                                          double* __restrict__ out_rows) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long rr = warp; rr < rows; rr += nwarps) {
        const int i = src_lo + (int)rr;
        const uint16_t* drow = D + rr * ld;
        double xi[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) xi[c] = c < dim ? (double)__ldg(X + (size_t)i * dim + c) : 0.0;
        double acc = 0.0;
        for (int j = lane; j < n; j += 32) {
            if (j == i) continue;
            const unsigned dij = drow[j];
            if (dij == kDistInf) {
                acc += 1.0;
                continue;
            }
            // |X_i - X_j|^2 exactly enough in FP64 (the difference of two floats is exact there)
            double sq = 0.0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < dim) {
                    const double dx = xi[c] - (double)__ldg(X + (size_t)j * dim + c);
                    sq = fma(dx, dx, sq);
                }
            }
            // its square root: FP32, refined by one Newton step on the FP64 residual
            double x = 0.0;
            if (sq > 0.0) {
                const float x0 = sqrtf((float)sq);
                const double res = fma(-(double)x0, (double)x0, sq);
                x = (double)x0 + (double)((float)res / (2.0f * x0));
            }
            // d - x in FP64 (it cancels when the drawing is good), the rest in FP32
            const float t = (float)((double)dij - x) / (float)dij;
            acc += (double)(t * t);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) out_rows[i] = acc;
    }
}

// Sum of vals[0 .. count) into *out in a fixed order (one CTA): thread t sums
// t, t + 1024, ...; then a tree over the threads.
__global__ void __launch_bounds__(1024) sum_kernel(const double* __restrict__ vals, long long count, double scale,
                                                   double* __restrict__ out) {
    __shared__ double s[1024];
    double a = 0.0;
    for (long long i = threadIdx.x; i < count; i += 1024) a += vals[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] * scale;
}

}  // namespace

size_t np_smem_bytes(int32_t n) { return 3 * (size_t)((n + 31) / 32) * sizeof(uint32_t); }

cudaError_t launch_np(const int32_t* row_ptr, const int32_t* col, int32_t n, const float* X, int32_t dim, int32_t r,
                      int32_t* out_c, int32_t* out_inter, double* term, double* out_sum, cudaStream_t s) {
    const size_t smem = np_smem_bytes(n);
    cudaError_t e = cudaFuncSetAttribute(np_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = n < device_sm_count() * 8 ? n : device_sm_count() * 8;
    np_kernel<<<grid, kNpThreads, smem, s>>>(row_ptr, col, n, X, dim, r, out_c, out_inter, term);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sum_kernel<<<1, 1024, 0, s>>>(term, n, 1.0, out_sum);
    return cudaGetLastError();
}

cudaError_t launch_stress_rows(const uint16_t* D, long long ld, int32_t rows, int32_t src_lo, int32_t n,
                               const float* X, int32_t dim, double* out_rows, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    long long g = ((long long)rows * 32 + 255) / 256;
    if (g > device_sm_count() * 16ll) g = device_sm_count() * 16ll;
    stress_rows_kernel<<<(unsigned)g, 256, 0, s>>>(D, ld, rows, src_lo, n, X, dim, out_rows);
    return cudaGetLastError();
}

cudaError_t launch_sum(const double* vals, long long count, double scale, double* out, cudaStream_t s) {
    sum_kernel<<<1, 1024, 0, s>>>(vals, count, scale, out);
    return cudaGetLastError();
}

}  // namespace gumap
