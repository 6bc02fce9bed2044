// Device-side validation of a CSR graph given by device pointers: the input
// of the method is an undirected unweighted graph G = (V, E) (Algorithm 1,
// Algorithm 4 input), so every row must be strictly ascending (no duplicate
// edge), free of self loops, with ids in [0, n), and (u, v) present iff
// (v, u) present. One thread per row; symmetry is a binary search of u in
// the row of each neighbour v.
#include "gumap_internal.cuh"

namespace gumap {

namespace {

__global__ void validate_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                                int64_t nnz, int32_t* bad) {
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (long long)gridDim.x * blockDim.x) {
        const int b = rp[u], e = rp[u + 1];
        if (u == 0 && b != 0) { atomicOr(bad, 1); continue; }
        if (u == n - 1 && (int64_t)e != nnz) { atomicOr(bad, 1); continue; }
        if (e < b || b < 0 || (int64_t)e > nnz) { atomicOr(bad, 1); continue; }
        int prev = -1;
        for (int p = b; p < e; ++p) {
            const int v = col[p];
            if (v < 0 || v >= n || v == u || v <= prev) { atomicOr(bad, 1); break; }
            prev = v;
            int lo = rp[v], hi = rp[v + 1];
            if (lo < 0 || hi > nnz || hi < lo) { atomicOr(bad, 1); break; }
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (col[mid] < u) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= rp[v + 1] || col[lo] != u) { atomicOr(bad, 1); break; }
        }
    }
}

}  // namespace

cudaError_t launch_validate_csr(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, int32_t* bad,
                                cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
    if (e != cudaSuccess || n <= 0) return e;
    long long g = ((long long)n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    validate_kernel<<<(unsigned)g, 256, 0, s>>>(row_ptr, col, n, nnz, bad);
    return cudaGetLastError();
}

}  // namespace gumap
