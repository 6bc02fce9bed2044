// Device-side validation of a CSR graph given by device pointers: the input
// of the method is an undirected unweighted graph G = (V, E) (Algorithm 1,
// Algorithm 4 input), so every row must be strictly ascending (no duplicate
// edge), free of self loops, with ids in [0, n), and (u, v) present iff
// (v, u) present. Row bounds are checked one thread per row; every edge is
// checked by its own thread (its row found by a binary search of row_ptr,
// the reverse edge by a binary search of the neighbour's row), so a hub's
// row costs no more time than any other.
#include "gumap_internal.cuh"

namespace gumap {

namespace {

__global__ void validate_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int32_t n,
                                int64_t nnz, int32_t* bad) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long u = tid; u < n; u += nthr) {
        const int b = rp[u], e = rp[u + 1];
        if ((u == 0 && b != 0) || (u == n - 1 && (int64_t)e != nnz) || e < b || b < 0 || (int64_t)e > nnz)
            atomicOr(bad, 1);
    }
    for (long long p = tid; p < nnz; p += nthr) {
        // row u of edge p: the last u with rp[u] <= p (rows may be empty)
        int lo = 0, hi = n;  // invariant rp[lo] <= p, answer in [lo, hi)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if ((long long)rp[mid] <= p) lo = mid;
            else hi = mid;
        }
        const int u = lo;
        const int v = col[p];
        bool ok = v >= 0 && v < n && v != u;
        if (ok && p > rp[u]) ok = col[p - 1] < v;
        if (ok) {
            int a = rp[v], z = rp[v + 1];
            ok = a >= 0 && (int64_t)z <= nnz && z >= a;
            if (ok) {
                while (a < z) {
                    const int mid = (a + z) >> 1;
                    if (col[mid] < u) a = mid + 1;
                    else z = mid;
                }
                ok = a < rp[v + 1] && col[a] == u;
            }
        }
        if (!ok) atomicOr(bad, 1);
    }
}

}  // namespace

cudaError_t launch_validate_csr(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, int32_t* bad,
                                cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
    if (e != cudaSuccess || n <= 0) return e;
    const long long work = nnz > n ? nnz : (long long)n;
    long long g = (work + 255) / 256;
    if (g > device_sm_count() * 32ll) g = device_sm_count() * 32ll;
    validate_kernel<<<(unsigned)g, 256, 0, s>>>(row_ptr, col, n, nnz, bad);
    return cudaGetLastError();
}

}  // namespace gumap
