// Spectral layout of the kNN graph G_k: the initial coordinates of the
// layout stage ("initialize the coordinates in X using spectral layout",
// Algorithm 1; Section 3.2, after Koren's spectral graph drawing).
//
// With W the fuzzy-union weights of G_k and D = diag(W 1), Koren's
// degree-normalised eigenvectors solve L x = mu D x (L = D - W) for the
// smallest mu after the trivial mu = 0 (x constant), D-normalised. With
// y = D^(1/2) x they are the eigenvectors of M = D^(-1/2) W D^(-1/2) of the
// largest eigenvalues theta = 1 - mu after the trivial one, whose vector is
// t = D^(1/2) 1 / |D^(1/2) 1|.
//
// Lanczos iteration on M with t projected out (every product is followed by
// that projection), FP64 vectors kept as the columns of Q and reorthogonalised
// against all of them by classical Gram-Schmidt applied twice. Kernels: the
// product M q (one warp per row of the union graph's CSR), dot products and
// Q^T w (per-chunk partial sums reduced in a fixed order, so runs repeat
// bit for bit), w -= Q h, and the vector updates. The tridiagonal matrix of
// the recurrence is small (at most a few hundred rows) and is solved on the
// host: its largest eigenvalues by bisection on Sturm counts, their vectors
// by inverse iteration with a pivoted tridiagonal factorisation,
// orthogonalised within clusters of equal eigenvalues. A Ritz pair's
// residual is beta_j |s_last|. A Krylov space from one start vector holds
// one vector per distinct eigenvalue, so each run of Lanczos locks only its
// top Ritz vector once converged, and later runs project the locked vectors
// out as well: run r finds the r-th largest eigenvalue, copies of a repeated
// one included. A run whose basis fills first restarts from its current top
// Ritz vector. x = D^(-1/2) y for each locked y. Vertices with no edge keep
// coordinate 0 (the start vector is zero there, and M maps the rest to the
// rest).
#include "gumap.h"
#include "gumap_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace gumap {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kVecThreads = 256;
constexpr int kChunk = kSpectralChunk;  // rows per partial sum

struct SpecGraph {
    const unsigned long long* rowoff;  // [n + 1]
    const int32_t* col;
    const float* w;
    int32_t n;
};

// s_i = 1 / sqrt(d_i), d_i = sum_j w_ij (0 for a vertex with no edge); one warp per row
__global__ void degree_kernel(SpecGraph g, double* __restrict__ s, double* __restrict__ sq) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < g.n; i += nwarps) {
        double d = 0.0;
        for (unsigned long long e = g.rowoff[i] + lane; e < g.rowoff[i + 1]; e += 32) d += (double)g.w[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
        if (lane == 0) {
            s[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
            sq[i] = d > 0.0 ? sqrt(d) : 0.0;
        }
    }
}

// y = s . (W (s . x)) with z = s . x precomputed; one warp per row
__global__ void spmv_kernel(SpecGraph g, const double* __restrict__ s, const double* __restrict__ z,
                            double* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = warp; i < g.n; i += nwarps) {
        double acc = 0.0;
        for (unsigned long long e = g.rowoff[i] + lane; e < g.rowoff[i + 1]; e += 32)
            acc += (double)g.w[e] * z[g.col[e]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) y[i] = s[i] * acc;
    }
}

__global__ void mul_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] * b[i];
}

// part[j * chunks + c] = sum over rows r of chunk c of Q[j][r] * w[r], for j < m (blockIdx.y = j)
__global__ void dots_kernel(long long n, const double* __restrict__ Q, long long ld, int m,
                            const double* __restrict__ w, double* __restrict__ part, int chunks) {
    __shared__ double red[kVecThreads / 32];
    const int j = blockIdx.y;
    const long long r0 = (long long)blockIdx.x * kChunk;
    const double* q = Q + (long long)j * ld;
    double acc = 0.0;
    for (long long r = r0 + threadIdx.x; r < n && r < r0 + kChunk; r += kVecThreads) acc += q[r] * w[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kVecThreads / 32; ++i) t += red[i];
        part[(long long)j * chunks + blockIdx.x] = t;
    }
}

// out[j] = sum over c of part[j * chunks + c], in order (one thread per j)
__global__ void reduce_parts_kernel(const double* __restrict__ part, int chunks, int m, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double t = 0.0;
    for (int c = 0; c < chunks; ++c) t += part[(long long)j * chunks + c];
    out[j] = t;
}

// w -= sum_j h[j] Q[j] (h on the device), then optionally w *= mask (vertices with edges)
__global__ void gemv_sub_kernel(long long n, const double* __restrict__ Q, long long ld, int m,
                                const double* __restrict__ h, double* __restrict__ w) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        double acc = w[r];
        for (int j = 0; j < m; ++j) acc -= h[j] * Q[(long long)j * ld + r];
        w[r] = acc;
    }
}

// out = a * x + b * y (out may alias x or y)
__global__ void axpby_kernel(long long n, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, double* out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a * x[i] + b * y[i];
}

// start vector: a counter-based pseudo-random value per vertex (splitmix64 of
// the index and the run), zero where the vertex has no edge
__global__ void start_kernel(long long n, const double* __restrict__ s, double* __restrict__ q,
                             unsigned long long seed) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i + (seed + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        q[i] = s[i] > 0.0 ? u - 0.5 : 0.0;
    }
}

// X[r][c] = (float)(sign * s[r] * y[r]) for column c of a row-major [n][dim] output
__global__ void emit_kernel(long long n, const double* __restrict__ s, const double* __restrict__ y, double sign,
                            int c, int dim, float* __restrict__ X) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
        X[r * dim + c] = (float)(sign * s[r] * y[r]);
}

// CSR of the radix-built COO: rows from the sorted (row << B | col) keys
__global__ void radix_csr_kernel(const unsigned long long* __restrict__ keys, long long nnz, int key_bits, int n,
                                 unsigned long long* __restrict__ rowoff, int32_t* __restrict__ col) {
    const unsigned long long mask = (1ull << key_bits) - 1ull;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x)
        col[p] = (int32_t)(keys[p] & mask);
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = nnz;  // first entry of row r
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if ((long long)(keys[mid] >> key_bits) < r) lo = mid + 1;
            else hi = mid;
        }
        rowoff[r] = (unsigned long long)lo;
    }
}

// ---------------------------------------------------------------- host side

// eigenvalues of the symmetric tridiagonal T (diagonal a, off-diagonal b) below x
int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
    int cnt = 0;
    double q = 1.0;
    const size_t m = a.size();
    for (size_t i = 0; i < m; ++i) {
        const double off = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        q = (a[i] - x) - (i > 0 ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;  // x sits on an eigenvalue of the leading block: count it below
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// the r-th largest eigenvalue (r = 1 .. m), by bisection on Sturm counts
double tri_eigenvalue(const std::vector<double>& a, const std::vector<double>& b, int r) {
    const size_t m = a.size();
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < m; ++i) {  // Gershgorin bounds
        const double rad = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - rad);
        hi = std::max(hi, a[i] + rad);
    }
    const int below = (int)m - r;  // eigenvalues strictly below the wanted one
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (sturm_below(a, b, mid) > below) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// z solving (T - theta I) z = rhs by Gaussian elimination with partial
// pivoting on the tridiagonal matrix (the upper factor has two
// superdiagonals); a zero pivot is replaced by a tiny one, as inverse
// iteration wants
void tri_solve(const std::vector<double>& a, const std::vector<double>& b, double theta, std::vector<double>& rhs,
               double tiny) {
    const size_t m = a.size();
    std::vector<double> u0(m), u1(m, 0.0), u2(m, 0.0), y(m);
    double cd = a[0] - theta, cs = m > 1 ? b[0] : 0.0, cr = rhs[0];
    for (size_t i = 0; i + 1 < m; ++i) {
        const double sub = b[i], dn = a[i + 1] - theta, sn = i + 2 < m ? b[i + 1] : 0.0, rn = rhs[i + 1];
        if (std::fabs(cd) >= std::fabs(sub)) {
            if (cd == 0.0) cd = tiny;
            const double f = sub / cd;
            u0[i] = cd;
            u1[i] = cs;
            u2[i] = 0.0;
            y[i] = cr;
            cd = dn - f * cs;
            cs = sn;
            cr = rn - f * cr;
        } else {
            const double f = cd / sub;
            u0[i] = sub;
            u1[i] = dn;
            u2[i] = sn;
            y[i] = rn;
            const double nd = cs - f * dn, ns = -f * sn, nr = cr - f * rn;
            cd = nd;
            cs = ns;
            cr = nr;
        }
    }
    u0[m - 1] = cd == 0.0 ? tiny : cd;
    y[m - 1] = cr;
    for (size_t ii = m; ii-- > 0;) {
        double t = y[ii];
        if (ii + 1 < m) t -= u1[ii] * rhs[ii + 1];
        if (ii + 2 < m) t -= u2[ii] * rhs[ii + 2];
        rhs[ii] = t / u0[ii];
    }
}

// the `want` largest eigenpairs of T (vectors orthonormal, also within clusters)
void tri_top(const std::vector<double>& a, const std::vector<double>& b, int want, std::vector<double>& theta,
             std::vector<std::vector<double>>& vecs) {
    const size_t m = a.size();
    double scale = 0.0;
    for (size_t i = 0; i < m; ++i) scale = std::max(scale, std::fabs(a[i]) + (i ? std::fabs(b[i - 1]) : 0.0));
    const double tiny = std::max(scale, 1e-300) * 1e-15;
    theta.assign((size_t)want, 0.0);
    vecs.assign((size_t)want, std::vector<double>(m, 0.0));
    for (int r = 0; r < want; ++r) {
        theta[(size_t)r] = tri_eigenvalue(a, b, r + 1);
        std::vector<double>& z = vecs[(size_t)r];
        for (size_t i = 0; i < m; ++i) z[i] = 1.0 + 0.1 * std::sin(1.0 + 3.7 * (double)i + 1.3 * r);
        for (int it = 0; it < 4; ++it) {
            tri_solve(a, b, theta[(size_t)r], z, tiny);
            for (int q = 0; q < r; ++q)  // orthogonal to the pairs of (nearly) equal eigenvalue
                if (std::fabs(theta[(size_t)q] - theta[(size_t)r]) <= 1e-8 * std::max(scale, 1e-300)) {
                    double d = 0.0;
                    for (size_t i = 0; i < m; ++i) d += z[i] * vecs[(size_t)q][i];
                    for (size_t i = 0; i < m; ++i) z[i] -= d * vecs[(size_t)q][i];
                }
            double nrm = 0.0;
            for (double x : z) nrm += x * x;
            nrm = std::sqrt(nrm);
            if (nrm == 0.0) break;
            for (double& x : z) x /= nrm;
        }
    }
}

int grid_for(long long work, int threads, int cap) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

int spectral_layout(const SpectralInput& in, int dim, float* out_X, double* out_mu, gumap_spectral_info* info,
                    SpectralScratch& scr, cudaStream_t st) {
    const long long n = in.n;
    const int sms = device_sm_count();
    const int vgrid = grid_for(n, kVecThreads, sms * 16);
    const int wgrid = grid_for(n * 32, kVecThreads, sms * 16);
    SpecGraph g{in.rowoff, in.col, in.w, in.n};
    cudaError_t e;
#define SCK(call)                                       \
    do {                                                \
        if ((e = (call)) != cudaSuccess) return (int)e;  \
    } while (0)
    double* s = scr.s;      // D^(-1/2)
    double* sq = scr.sq;    // D^(1/2)
    double* t = scr.t;      // the trivial vector
    double* wv = scr.w;
    double* z = scr.z;
    double* Q = scr.Q;
    const long long ld = n;
    const int m_max = scr.m_max;
    const int chunks = (int)((n + kChunk - 1) / kChunk);
    double* part = scr.part;  // [(m_max + 1) * chunks]
    double* hdev = scr.h;     // [m_max + 1]

    degree_kernel<<<wgrid, kVecThreads, 0, st>>>(g, s, sq);
    SCK(cudaGetLastError());
    // dot products of columns [0, m) of a column-major block with w into hdev
    // (and to the host when `host` is given)
    auto dots = [&](const double* cols, int m, const double* w, double* host) -> cudaError_t {
        dots_kernel<<<dim3((unsigned)chunks, (unsigned)m), kVecThreads, 0, st>>>(n, cols, ld, m, w, part, chunks);
        reduce_parts_kernel<<<(m + 127) / 128, 128, 0, st>>>(part, chunks, m, hdev);
        cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess || !host) return e2;
        if ((e2 = cudaMemcpyAsync(host, hdev, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return e2;
        return cudaStreamSynchronize(st);
    };
    // w -= cols h for the first m columns (h on the device in hdev)
    auto sub = [&](const double* cols, int m, double* w) -> cudaError_t {
        gemv_sub_kernel<<<vgrid, kVecThreads, 0, st>>>(n, cols, ld, m, hdev, w);
        return cudaGetLastError();
    };
    double tn = 0.0;
    SCK(dots(sq, 1, sq, &tn));
    tn = std::sqrt(tn);
    if (!(tn > 0.0)) return -2;  // no edge at all
    axpby_kernel<<<vgrid, kVecThreads, 0, st>>>(n, 1.0 / tn, sq, 0.0, sq, t);
    SCK(cudaGetLastError());
    // project the trivial direction out of w (dots / sub leave the coefficient in hdev)
    auto deflate = [&](double* w) -> cudaError_t {
        cudaError_t e2 = dots(t, 1, w, nullptr);
        if (e2 != cudaSuccess) return e2;
        return sub(t, 1, w);
    };
    auto normalize_into = [&](const double* w, double* dst, double* nrm_out) -> cudaError_t {
        double nn = 0.0;
        cudaError_t e2 = dots(w, 1, w, &nn);
        if (e2 != cudaSuccess) return e2;
        const double nrm = std::sqrt(nn);
        *nrm_out = nrm;
        axpby_kernel<<<vgrid, kVecThreads, 0, st>>>(n, nrm > 0.0 ? 1.0 / nrm : 0.0, w, 0.0, w, dst);
        return cudaGetLastError();
    };

    // Runs of Lanczos, each locking one vector: the largest eigenvalue of M
    // with t and the vectors locked so far projected out. A Krylov space
    // holds one vector per distinct eigenvalue, so a repeated eigenvalue's
    // other copies are found by the runs after the first.
    const double tol = 1e-10;
    const int max_restarts = 30;
    int iters = 0, restarts = 0;
    double worst = 0.0;
    std::vector<double> al, be, theta_run, locked_theta;
    std::vector<std::vector<double>> vecs;
    double* Y = scr.Y;
    int nl = 0;  // locked vectors, the columns Y[0 .. nl)
    // project t and the locked vectors out of w
    auto deflate_all = [&](double* w) -> cudaError_t {
        cudaError_t e2 = deflate(w);
        if (e2 != cudaSuccess || nl == 0) return e2;
        if ((e2 = dots(Y, nl, w, nullptr)) != cudaSuccess) return e2;
        return sub(Y, nl, w);
    };
    bool out_of_space = false;
    for (int run = 0; nl < dim && !out_of_space; ++run) {
        start_kernel<<<vgrid, kVecThreads, 0, st>>>(n, s, wv, (unsigned long long)run);
        SCK(cudaGetLastError());
        bool locked = false;
        for (int rs = 0; !locked; ++rs) {
            SCK(deflate_all(wv));
            double nrm = 0.0;
            SCK(normalize_into(wv, Q, &nrm));
            if (!(nrm > 1e-12)) {  // nothing left outside the locked space
                out_of_space = true;
                break;
            }
            al.clear();
            be.clear();
            bool conv = false;
            double resid = 1e300;
            int j = 0;
            for (; j < m_max; ++j) {
                double* qj = Q + (long long)j * ld;
                mul_kernel<<<vgrid, kVecThreads, 0, st>>>(n, s, qj, z);
                spmv_kernel<<<wgrid, kVecThreads, 0, st>>>(g, s, z, wv);
                SCK(cudaGetLastError());
                double alpha = 0.0;
                SCK(dots(qj, 1, wv, &alpha));
                al.push_back(alpha);
                // full reorthogonalisation (it removes the alpha q_j and beta q_(j-1) parts too)
                for (int pass = 0; pass < 2; ++pass) {
                    SCK(dots(Q, j + 1, wv, nullptr));
                    SCK(sub(Q, j + 1, wv));
                }
                SCK(deflate_all(wv));
                ++iters;
                double bn = 0.0;
                SCK(dots(wv, 1, wv, &bn));
                const double beta = std::sqrt(bn);
                const bool exhausted = beta <= 1e-13;  // the Krylov space is invariant
                const bool last = j + 1 == m_max;
                if ((j + 1) % 8 == 0 || last || exhausted) {
                    tri_top(al, be, 1, theta_run, vecs);
                    resid = std::fabs(beta * vecs[0][(size_t)j]);
                    conv = resid <= tol || exhausted;
                }
                if (conv || last) {
                    ++j;
                    break;
                }
                be.push_back(beta);
                axpby_kernel<<<vgrid, kVecThreads, 0, st>>>(n, 1.0 / beta, wv, 0.0, wv, Q + (long long)(j + 1) * ld);
                SCK(cudaGetLastError());
            }
            // the top Ritz vector Q s into Y[nl]
            const int mused = j;
            SCK(cudaMemcpyAsync(hdev, vecs[0].data(), sizeof(double) * (size_t)mused, cudaMemcpyHostToDevice, st));
            double* y = Y + (long long)nl * ld;
            SCK(cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n, st));
            SCK(sub(Q, mused, y));  // y = -Q s
            axpby_kernel<<<vgrid, kVecThreads, 0, st>>>(n, -1.0, y, 0.0, y, y);
            SCK(cudaGetLastError());
            SCK(cudaStreamSynchronize(st));
            if (conv || rs >= max_restarts) {
                locked_theta.push_back(theta_run[0]);
                worst = std::max(worst, resid);
                ++nl;
                locked = true;
            } else {  // restart from the current Ritz vector
                ++restarts;
                SCK(cudaMemcpyAsync(wv, y, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st));
            }
        }
    }
    const int have = nl;
    // x = D^(-1/2) y, sign: the entry of largest magnitude positive (first such index)
    std::vector<double> host_y((size_t)n);
    for (int r = 0; r < dim; ++r) {
        double sign = 1.0;
        if (r < have) {
            // y_r lives in scr.Y; x = s . y
            mul_kernel<<<vgrid, kVecThreads, 0, st>>>(n, s, scr.Y + (long long)r * ld, z);
            SCK(cudaGetLastError());
            SCK(cudaMemcpyAsync(host_y.data(), z, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
            SCK(cudaStreamSynchronize(st));
            long long arg = 0;
            double best = -1.0;
            for (long long i = 0; i < n; ++i)
                if (std::fabs(host_y[(size_t)i]) > best) {
                    best = std::fabs(host_y[(size_t)i]);
                    arg = i;
                }
            if (host_y[(size_t)arg] < 0.0) sign = -1.0;
            emit_kernel<<<vgrid, kVecThreads, 0, st>>>(n, s, scr.Y + (long long)r * ld, sign, r, dim, out_X);
            if (out_mu) out_mu[r] = 1.0 - locked_theta[(size_t)r];
        } else {
            SCK(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)n, st));
            emit_kernel<<<vgrid, kVecThreads, 0, st>>>(n, s, z, 1.0, r, dim, out_X);
            if (out_mu) out_mu[r] = NAN;
        }
        SCK(cudaGetLastError());
    }
    SCK(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = iters;
        info->restarts = restarts;
        info->residual = worst;
        info->converged = worst <= tol ? 1 : 0;
    }
#undef SCK
    return 0;
}

cudaError_t launch_radix_csr(const unsigned long long* keys, long long nnz, int key_bits, int32_t n,
                             unsigned long long* rowoff, int32_t* col, cudaStream_t s) {
    const long long work = std::max<long long>(nnz, (long long)n + 1);
    radix_csr_kernel<<<grid_for(work, 256, device_sm_count() * 16), 256, 0, s>>>(keys, nnz, key_bits, n, rowoff, col);
    return cudaGetLastError();
}

}  // namespace gumap
