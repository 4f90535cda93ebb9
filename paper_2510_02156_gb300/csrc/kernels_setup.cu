// kernels_setup.cu -- setup of ROR-BK (Algorithm 1's set-up, Section 3.1).
//
//   k_validate_csr        structure and finiteness checks of the copied A
//   k_block_transpose     per static block: nonzeros sorted by (column, row),
//                         distinct-column segments, coupled rows
//   k_centroid_*          centroids Abar_t (sum of the block's rows), the Gram
//                         Abar Abar^T one row per warp, C's row sums
//   k_proposal            Pbar_t = exp(-2 sum_j C(t,j) / n) and its running sum
//   k_static_ops          W_t = (A_t A_t^T + mu I)^{-1} per block through a
//                         Cholesky factor, on the block's coupled rows only
//
// The "coupled" rows of a row set are those sharing at least one column with
// another row of the set.  The Gram A_t A_t^T is diagonal outside the
// coupled rows, so the Cholesky factor, its inverse and W_t are too; the dense
// work is restricted to the coupled rows, which gives the same numbers as the
// dense factorisation (zero multipliers contribute exact zeros).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace rorbk {

// ------------------------------------------------------------------ checks
__global__ void k_validate_csr(const int *__restrict__ rowptr, const int *__restrict__ col,
                               const double *__restrict__ val, int m, int n, int *flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        int p0 = rowptr[i], p1 = rowptr[i + 1];
        if (p1 < p0) { atomicOr(flags, 1); continue; }
        int prev = -1;
        for (int p = p0; p < p1; ++p) {
            int c = col[p];
            if (c < 0 || c >= n || c <= prev) { atomicOr(flags, 1); break; }
            prev = c;
            if (!isfinite(val[p])) atomicOr(flags, 2);
        }
    }
}

__global__ void k_widen(const float *__restrict__ in, double *__restrict__ out, long long nn) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

__global__ void k_narrow(const double *__restrict__ in, float *__restrict__ out, long long nn) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// First entry of every block: rowptr[off[t]], t = 0..k.
__global__ void k_block_nz(const int *__restrict__ rowptr, const int *__restrict__ off, int k,
                           int *__restrict__ out) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= k; t += gridDim.x * blockDim.x)
        out[t] = rowptr[off[t]];
}

// ---------------------------------------------------------- block transpose
// One block of threads per static block t.  Entry p of the block's CSR range
// lands at rank(p) = #entries with a smaller column + #entries in earlier
// rows with the same column, found by binary searches in every row of the
// block (rows hold ascending columns).
__device__ __forceinline__ int lower_bound_col(const int *col, int lo, int hi, int c) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_block_transpose(const int *__restrict__ rowptr, const int *__restrict__ col,
                                  const double *__restrict__ val, const int *__restrict__ off,
                                  int *__restrict__ bt_col, uint16_t *__restrict__ bt_row,
                                  double *__restrict__ bt_val, uint16_t *__restrict__ bt_off,
                                  int *__restrict__ bt_seg,
                                  int *__restrict__ nseg_out, unsigned char *__restrict__ coupled,
                                  int *__restrict__ ncoupled_out) {
    __shared__ int scan_scratch[33];
    __shared__ unsigned char flag[kMaxBlockRows];
    const int t = blockIdx.x;
    const int r0 = off[t], r1 = off[t + 1], s = r1 - r0;
    const int p0 = rowptr[r0], E = rowptr[r1] - p0;
    for (int a = threadIdx.x; a < s; a += blockDim.x) flag[a] = 0;

    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        int p = p0 + e;
        int c = col[p];
        int lo = r0, hi = r1;                    // row of entry p: last i with rowptr[i] <= p
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (rowptr[mid] <= p) lo = mid; else hi = mid;
        }
        int a = lo - r0;
        int rank = 0;
        for (int b = 0; b < s; ++b) {
            int q0 = rowptr[r0 + b], q1 = rowptr[r0 + b + 1];
            int lb = lower_bound_col(col, q0, q1, c);
            rank += lb - q0;
            if (b < a && lb < q1 && col[lb] == c) rank += 1;
        }
        int dst = p0 + rank;
        bt_col[dst] = c;
        bt_row[dst] = (uint16_t)a;
        bt_val[dst] = val[p];
        bt_off[dst] = (uint16_t)e;
    }
    __syncthreads();

    int nseg = 0;
    for (int base = 0; base < E; base += blockDim.x) {
        int q = base + threadIdx.x;
        int head = 0;
        if (q < E) head = (q == 0) || (bt_col[p0 + q] != bt_col[p0 + q - 1]);
        int total;
        int pre = block_exclusive_scan(head, scan_scratch, &total);
        if (head) {
            bt_seg[p0 + nseg + pre] = p0 + q;
            int c = bt_col[p0 + q];
            int e = q + 1;
            while (e < E && bt_col[p0 + e] == c) ++e;
            if (e - q > 1)
                for (int u = q; u < e; ++u) flag[bt_row[p0 + u]] = 1;
        }
        nseg += total;
    }
    __syncthreads();
    int cnt = 0;
    for (int a = threadIdx.x; a < s; a += blockDim.x) {
        coupled[r0 + a] = flag[a];
        cnt += flag[a];
    }
    int tot = block_sum(cnt, scan_scratch);
    if (threadIdx.x == 0) {
        nseg_out[t] = nseg;
        ncoupled_out[t] = tot;
    }
}

// A dense A (every entry stored, rows of n entries): block t's column-sorted
// copy is its transpose -- segment c holds rows 0 .. s-1 of column c in order --
// and every row of a block with two or more rows shares a column with another
// (all are coupled).  The same arrays as k_block_transpose, formed by a
// grid-wide transpose instead of one block of threads ranking every entry
// (which costs s binary searches per entry: minutes for 256 x 100,000 blocks).
__global__ void k_block_transpose_dense(const double *__restrict__ val, const int *__restrict__ off,
                                        int n, int *__restrict__ bt_col, uint16_t *__restrict__ bt_row,
                                        double *__restrict__ bt_val, uint16_t *__restrict__ bt_off,
                                        int *__restrict__ bt_seg,
                                        int *__restrict__ nseg_out, unsigned char *__restrict__ coupled,
                                        int *__restrict__ ncoupled_out) {
    const int t = blockIdx.y;
    const int r0 = off[t], s = off[t + 1] - r0;
    const long long p0 = (long long)r0 * n, E = (long long)s * n;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long gs = (long long)gridDim.x * blockDim.x;
    for (long long d = gt; d < E; d += gs) {
        const long long c = d / s;
        const int a = (int)(d - c * s);
        bt_col[p0 + d] = (int)c;
        bt_row[p0 + d] = (uint16_t)a;
        bt_val[p0 + d] = val[p0 + (long long)a * n + c];
        bt_off[p0 + d] = (uint16_t)((long long)a * n + c);
    }
    for (long long c = gt; c < n; c += gs) bt_seg[p0 + c] = (int)(p0 + c * s);
    for (long long a = gt; a < s; a += gs) coupled[r0 + a] = s > 1 ? 1 : 0;
    if (gt == 0) {
        nseg_out[t] = n;
        ncoupled_out[t] = s > 1 ? s : 0;
    }
}

// The Gram of every static block of a dense A on its coupled rows (all of
// them): G_ij = sum over ascending columns of a_ic a_jc, one fused chain from
// 0 (k_static_ops' merge of two dense rows visits the same columns in the same
// order), mu added to the diagonal.  Grid (tiles of kSgT x kSgT entries of
// the lower triangle, blocks); the rows' next kSgC columns are staged in
// shared memory.  k_static_ops then factors the block without forming G.
constexpr int kSgT = 16, kSgC = 64;
__global__ void __launch_bounds__(kSgT * kSgT) k_dense_static_gram(const double *__restrict__ val,
                                                                   const int *__restrict__ off, int n,
                                                                   double mu,
                                                                   const long long *__restrict__ w_ptr,
                                                                   double *__restrict__ w_ss) {
    __shared__ double sa[kSgT][kSgC + 1], sb[kSgT][kSgC + 1];
    const int t = blockIdx.y;
    const int r0 = off[t], s = off[t + 1] - r0;
    if (s < 2) return;                          // no coupled rows: W_t is diagonal
    const int nt = (s + kSgT - 1) / kSgT;
    int q = blockIdx.x, ti = 0;                 // tile (ti, tj), tj <= ti
    if (q >= nt * (nt + 1) / 2) return;
    while (q > ti) { q -= ti + 1; ++ti; }
    const int tj = q, tid = threadIdx.x;
    const int ta = tid / kSgT, tb = tid % kSgT;
    const int a = ti * kSgT + ta, b = tj * kSgT + tb;
    double acc = 0.0;
    for (int c0 = 0; c0 < n; c0 += kSgC) {
        const int w = min(kSgC, n - c0);
        for (int e = tid; e < kSgT * kSgC; e += blockDim.x) {
            const int rr = e / kSgC, cc = e % kSgC;
            const int ra = ti * kSgT + rr, rb = tj * kSgT + rr;
            sa[rr][cc] = (ra < s && cc < w) ? val[(long long)(r0 + ra) * n + c0 + cc] : 0.0;
            sb[rr][cc] = (rb < s && cc < w) ? val[(long long)(r0 + rb) * n + c0 + cc] : 0.0;
        }
        __syncthreads();
        if (a < s && b <= a)
            for (int cc = 0; cc < w; ++cc) acc = __fma_rn(sa[ta][cc], sb[tb][cc], acc);
        __syncthreads();
    }
    if (a < s && b <= a) w_ss[w_ptr[t] + (long long)a * s + b] = a == b ? __dadd_rn(acc, mu) : acc;
}

// ||A_i||^2 of every row, one fused chain over the row's stored entries in
// order from 0: the dynamic update's Gram diagonal (before mu), formed once
// here instead of in every dynamic update (the same operations in the same
// order, so the same numbers).  V: the stored values the iteration reads.
template <typename V>
__global__ void k_row_norms(const int *__restrict__ rowptr, const V *__restrict__ val, int m,
                            double *__restrict__ rn) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double g = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const double v = (double)val[p];
            g = __fma_rn(v, v, g);
        }
        rn[i] = g;
    }
}

// ------------------------------------------------------------ device scans
// Exclusive scan of n ints in place (n < 2^31), three launches.
__global__ void k_scan_tiles(const int *__restrict__ in, int *__restrict__ out,
                             int *__restrict__ tile_sums, long long n) {
    __shared__ int sc[33];
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int v = i < n ? in[i] : 0;
    int total;
    int pre = block_exclusive_scan(v, sc, &total);
    if (i < n) out[i] = pre;
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}
__global__ void k_scan_sums(int *tile_sums, int ntiles, int *grand_total) {
    __shared__ int sc[33];
    int carry = 0;
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = i < ntiles ? tile_sums[i] : 0;
        int total;
        int pre = block_exclusive_scan(v, sc, &total);
        if (i < ntiles) tile_sums[i] = carry + pre;
        carry += total;
    }
    if (threadIdx.x == 0) *grand_total = carry;
}
__global__ void k_scan_add(int *out, const int *tile_sums, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[blockIdx.x];
}

// ------------------------------------------------------- centroids and C
// Centroid entry of block t at segment g: column bt_col[seg], value = sum of
// the segment's values in ascending row order (the rows are added in order).
__global__ void k_centroid_count(const int *__restrict__ rowptr, const int *__restrict__ off,
                                 const int *__restrict__ bt_col, const int *__restrict__ bt_seg,
                                 const int *__restrict__ nseg, int k, int *__restrict__ colcnt) {
    for (int t = blockIdx.x; t < k; t += gridDim.x) {
        int p0 = rowptr[off[t]];
        for (int g = threadIdx.x; g < nseg[t]; g += blockDim.x)
            atomicAdd(&colcnt[bt_col[bt_seg[p0 + g]]], 1);
    }
}

__device__ __forceinline__ double segment_sum(const double *bt_val, const int *bt_col,
                                              int q, int qend) {
    int c = bt_col[q];
    double v = 0.0;
    for (int u = q; u < qend && bt_col[u] == c; ++u) v = __dadd_rn(v, bt_val[u]);
    return v;
}

__global__ void k_centroid_fill(const int *__restrict__ rowptr, const int *__restrict__ off,
                                const int *__restrict__ bt_col, const double *__restrict__ bt_val,
                                const int *__restrict__ bt_seg, const int *__restrict__ nseg, int k,
                                const int *__restrict__ colptr, int *__restrict__ fill,
                                int *__restrict__ cb, double *__restrict__ cv) {
    for (int t = blockIdx.x; t < k; t += gridDim.x) {
        int p0 = rowptr[off[t]], pend = rowptr[off[t + 1]];
        for (int g = threadIdx.x; g < nseg[t]; g += blockDim.x) {
            int q = bt_seg[p0 + g];
            int c = bt_col[q];
            double v = segment_sum(bt_val, bt_col, q, pend);
            int pos = colptr[c] + atomicAdd(&fill[c], 1);
            cb[pos] = t;
            cv[pos] = v;
        }
    }
}

// Row t of G = Abar Abar^T, one warp per block t: columns c of Abar_t in
// ascending order, G(t, j) += Abar_tc * Abar_jc over the blocks j of column c
// (distinct j inside one column, so the lanes never collide).
__global__ void k_centroid_gram(const int *__restrict__ rowptr, const int *__restrict__ off,
                                const int *__restrict__ bt_col, const double *__restrict__ bt_val,
                                const int *__restrict__ bt_seg, const int *__restrict__ nseg,
                                int k, const int *__restrict__ colptr,
                                const int *__restrict__ cb, const double *__restrict__ cv,
                                double *__restrict__ G) {
    int lane = threadIdx.x & 31;
    int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= k) return;
    int p0 = rowptr[off[t]], pend = rowptr[off[t + 1]];
    double *Gt = G + (long long)t * k;
    for (int g = 0; g < nseg[t]; ++g) {
        int q = bt_seg[p0 + g];
        int c = bt_col[q];
        double v = segment_sum(bt_val, bt_col, q, pend);
        for (int e = colptr[c] + lane; e < colptr[c + 1]; e += 32) {
            int j = cb[e];
            Gt[j] = __fma_rn(v, cv[e], Gt[j]);
        }
        __syncwarp();
    }
}

// Dense centroids: Abar (k x n) row t = sum of the block's rows in order.
__global__ void k_centroid_dense(const double *__restrict__ A, long long ld,
                                 const int *__restrict__ off, int k, int n,
                                 double *__restrict__ Abar) {
    for (int t = blockIdx.y; t < k; t += gridDim.y)
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
            double v = 0.0;
            for (int i = off[t]; i < off[t + 1]; ++i) v = __dadd_rn(v, A[(long long)i * ld + c]);
            Abar[(long long)t * n + c] = v;
        }
}

// G = Abar Abar^T for dense centroids: one thread per (t, j), ascending c.
__global__ void k_centroid_gram_dense(const double *__restrict__ Abar, int k, int n,
                                      double *__restrict__ G) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int t = blockIdx.y;
    if (j >= k) return;
    const double *a = Abar + (long long)t * n, *b = Abar + (long long)j * n;
    double s = 0.0;
    for (int c = 0; c < n; ++c) s = __fma_rn(a[c], b[c], s);
    G[(long long)t * k + j] = s;
}

// sum_j C(t, j), C(t,t) = 1, C(t,j) = 0 when either centroid is zero.
__global__ void k_crowsum(const double *__restrict__ G, int k, double *__restrict__ rowsum) {
    int lane = threadIdx.x & 31;
    int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= k) return;
    double nt = sqrt(G[(long long)t * k + t]);
    double s = 0.0;
    for (int j = lane; j < k; j += 32) {
        double nj = sqrt(G[(long long)j * k + j]);
        double cij;
        if (j == t) cij = 1.0;
        else if (nt == 0.0 || nj == 0.0) cij = 0.0;
        else cij = fabs(G[(long long)t * k + j]) / (nt * nj);
        s += cij;
    }
    s = warp_sum(s);
    if (lane == 0) rowsum[t] = s;
}

// Pbar_t = exp(-2 rowsum_t / n); cdf_t = Pbar_0 + ... + Pbar_t summed in
// order by one thread (the normalisation of P is folded into the sampler).
__global__ void k_proposal(const double *__restrict__ rowsum, int k, double n,
                           double *__restrict__ cdf, double *__restrict__ pbar) {
    for (int t = threadIdx.x; t < k; t += blockDim.x) {
        const double v = exp(-2.0 * rowsum[t] / n);
        cdf[t] = v;
        pbar[t] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int t = 0; t < k; ++t) {
            s += cdf[t];
            cdf[t] = s;
        }
    }
}

// W = (L L^T)^{-1} from the Cholesky factor L in G (nS x nS row-major, lower),
// written over G (full, symmetric); Li is nS x nS scratch.  Linv column by
// column: Linv_jj = 1/L_jj, Linv_ij = -(sum_{c=j}^{i-1} L_ic Linv_cj) / L_ii, c
// ascending; then W_ij = sum_{c >= max(i,j)} Linv_ci Linv_cj (c ascending).
// All threads of the block take part.
__device__ void spd_inverse_from_factor(double *G, double *Li, int nS) {
    for (int j = threadIdx.x; j < nS; j += blockDim.x) {
        for (int i = 0; i < j; ++i) Li[(long long)i * nS + j] = 0.0;
        Li[(long long)j * nS + j] = 1.0 / G[(long long)j * nS + j];
        for (int i = j + 1; i < nS; ++i) {
            double acc = 0.0;
            for (int c = j; c < i; ++c)
                acc = __fma_rn(G[(long long)i * nS + c], Li[(long long)c * nS + j], acc);
            Li[(long long)i * nS + j] = -acc / G[(long long)i * nS + i];
        }
    }
    __syncthreads();
    for (long long idx = threadIdx.x; idx < (long long)nS * nS; idx += blockDim.x) {
        int i = (int)(idx / nS), j = (int)(idx % nS);
        if (j > i) continue;
        double acc = 0.0;
        for (int c = i; c < nS; ++c)
            acc = __fma_rn(Li[(long long)c * nS + i], Li[(long long)c * nS + j], acc);
        // the factor's (i, j) is read by nobody after the Linv pass
        G[(long long)i * nS + j] = acc;
    }
    __syncthreads();
    for (long long idx = threadIdx.x; idx < (long long)nS * nS; idx += blockDim.x) {
        int i = (int)(idx / nS), j = (int)(idx % nS);
        if (j > i) G[(long long)i * nS + j] = G[(long long)j * nS + i];
    }
}

// ------------------------------------------------------------ static ops
// One block of threads per static block t.  Inputs: the block's coupled
// flags and S offsets; outputs W on S (row-major |S|^2 at w_ss + w_ptr[t]),
// W_ii for uncoupled rows, and s_idx / s_pos.  Linv scratch has the layout of
// w_ss.
__global__ void k_static_ops(const int *__restrict__ rowptr, const int *__restrict__ col,
                             const double *__restrict__ val, const int *__restrict__ off,
                             double mu, const unsigned char *__restrict__ coupled,
                             const int *__restrict__ s_ptr, const long long *__restrict__ w_ptr,
                             uint16_t *__restrict__ s_idx, int *__restrict__ s_pos,
                             double *__restrict__ w_ss, double *__restrict__ w_diag,
                             double *__restrict__ linv, const long long *__restrict__ wood_ptr,
                             int *__restrict__ status, int gram_ready) {
    __shared__ int scan_scratch[33];
    __shared__ int bad;
    __shared__ double gdiag[kMaxBlockRows];
    const int t = blockIdx.x;
    const int r0 = off[t], s = off[t + 1] - r0;
    if (wood_ptr && wood_ptr[t] >= 0) {          // the n x n form serves this block
        for (int a = threadIdx.x; a < s; a += blockDim.x) {
            s_pos[r0 + a] = -1;
            w_diag[r0 + a] = 0.0;
        }
        return;
    }
    const int sb = s_ptr[t], nS = s_ptr[t + 1] - sb;
    double *G = w_ss + w_ptr[t];
    double *Li = linv + w_ptr[t];
    if (threadIdx.x == 0) bad = 0;

    // coupled rows in ascending order; diagonal of the Gram for every row
    int cnt = 0;
    for (int base = 0; base < s; base += blockDim.x) {
        int a = base + threadIdx.x;
        int f = a < s ? coupled[r0 + a] : 0;
        int total;
        int pre = block_exclusive_scan(f, scan_scratch, &total);
        if (a < s) {
            s_pos[r0 + a] = f ? cnt + pre : -1;
            if (f) s_idx[sb + cnt + pre] = (uint16_t)a;
            int p0 = rowptr[r0 + a], p1 = rowptr[r0 + a + 1];
            double g = 0.0;
            for (int p = p0; p < p1; ++p) g = __fma_rn(val[p], val[p], g);
            g = __dadd_rn(g, mu);
            gdiag[a] = g;
            if (!f) {
                if (!(g > 0.0)) { bad = 1; g = 1.0; }
                double li = 1.0 / sqrt(g);
                w_diag[r0 + a] = __dmul_rn(li, li);
            } else {
                w_diag[r0 + a] = 0.0;
            }
        }
        cnt += total;
    }
    __syncthreads();
    if (nS > 0) {
        // G on S: merges of the coupled rows (lower triangle + diagonal),
        // unless k_dense_static_gram formed it already (gram_ready)
        long long pairs = gram_ready ? 0 : (long long)nS * (nS + 1) / 2;
        for (long long idx = threadIdx.x; idx < pairs; idx += blockDim.x) {
            int i = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
            while ((long long)(i + 1) * (i + 2) / 2 <= idx) ++i;
            while ((long long)i * (i + 1) / 2 > idx) --i;
            int j = (int)(idx - (long long)i * (i + 1) / 2);
            int a = s_idx[sb + i], b = s_idx[sb + j];
            double g;
            if (i == j) g = gdiag[a];
            else g = row_merge_dot(col, val, rowptr[r0 + a], rowptr[r0 + a + 1],
                                   rowptr[r0 + b], rowptr[r0 + b + 1]);
            G[(long long)i * nS + j] = g;
        }
        __syncthreads();
        block_cholesky(G, nS, nS, &bad);
        spd_inverse_from_factor(G, Li, nS);
    }
    __syncthreads();
    if (threadIdx.x == 0 && bad) set_status(status, kDevNotSpd);
}

// ------------------------------------------------- the s >= n operators
// Lemma 1 and Section 3.1: a block with at least as many rows as A has columns
// stores V_t = (A_t^T A_t + mu I)^{-1} (n x n row-major at wood + wood_ptr[t])
// instead of W_t.  One block of threads per static block; blocks without the
// form return.  G_cd is the sum over the block's rows, ascending, of
// a_rc a_rd where both are stored: the merge of the two columns' segments of
// the column-sorted copy (rows ascending in each), one fused chain from 0;
// then mu on the diagonal, the Cholesky factor and the explicit inverse as for
// W_t.  linv has the layout of wood.
__global__ void k_wood_ops(const int *__restrict__ rowptr, const int *__restrict__ off, int n, double mu,
                           const long long *__restrict__ wood_ptr, const int *__restrict__ bt_col,
                           const uint16_t *__restrict__ bt_row, const double *__restrict__ bt_val,
                           double *__restrict__ wood, double *__restrict__ linv, int *__restrict__ status) {
    __shared__ int seg[kMaxBlockRows];         // n <= s <= kMaxBlockRows
    __shared__ int bad;
    const int t = blockIdx.x;
    const long long wp = wood_ptr[t];
    if (wp < 0) return;
    const int r0 = off[t], s = off[t + 1] - r0;
    const int p0 = rowptr[r0], pend = rowptr[r0 + s];
    double *G = wood + wp, *Li = linv + wp;
    if (threadIdx.x == 0) bad = 0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const int lo = lower_bound_col(bt_col, p0, pend, c);
        seg[c] = (lo < pend && bt_col[lo] == c) ? lo : -1;
    }
    __syncthreads();
    const long long pairs = (long long)n * (n + 1) / 2;
    for (long long idx = threadIdx.x; idx < pairs; idx += blockDim.x) {
        int i = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
        while ((long long)(i + 1) * (i + 2) / 2 <= idx) ++i;
        while ((long long)i * (i + 1) / 2 > idx) --i;
        const int j = (int)(idx - (long long)i * (i + 1) / 2);
        double g = 0.0;
        int p = seg[i], q = seg[j];
        if (p >= 0 && q >= 0) {
            while (p < pend && q < pend && bt_col[p] == i && bt_col[q] == j) {
                const int ri = bt_row[p], rj = bt_row[q];
                if (ri == rj) {
                    g = __fma_rn(bt_val[p], bt_val[q], g);
                    ++p;
                    ++q;
                } else if (ri < rj) {
                    ++p;
                } else {
                    ++q;
                }
            }
        }
        if (i == j) g = __dadd_rn(g, mu);
        G[(long long)i * n + j] = g;
    }
    __syncthreads();
    block_cholesky(G, n, n, &bad);
    spd_inverse_from_factor(G, Li, n);
    __syncthreads();
    if (threadIdx.x == 0 && bad) set_status(status, kDevNotSpd);
}

// FP64 working copy of FP32-stored values (exact), or FP32 copy of FP64
// values for the mixed-precision inner solve.
void widen_values(rorbk_ctx *h, int dtype) {
    const int gs = std::max(1, std::min(8 * h->num_sms, (int)((h->nnz + 255) / 256)));
    if (h->nnz == 0) return;
    if (dtype == RORBK_F32) k_widen<<<gs, 256, 0, h->stream>>>(h->val32, h->val, h->nnz);
    else if (h->val32) k_narrow<<<gs, 256, 0, h->stream>>>(h->val, h->val32, h->nnz);
}

// SELL-32 copy of A: lane l of slice s holds row sell_row[32 s + l]; entry j
// of that lane sits at ptr[s] + 32 j + l (the values of a dense A: grouped
// VW consecutive entries per lane, see below).
__global__ void k_sell_fill(const int *__restrict__ rowptr, const int *__restrict__ col,
                            const double *__restrict__ val, const float *__restrict__ val32,
                            int nslices, const long long *__restrict__ ptr,
                            const int *__restrict__ srow, const int *__restrict__ srlen,
                            int *__restrict__ scol, double *__restrict__ sval,
                            float *__restrict__ sval32, int dense) {
    const long long slot = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (slot >= (long long)nslices * 32) return;
    const int s = (int)(slot >> 5), lane = (int)(slot & 31);
    const int r = srow[slot], len = srlen[slot];
    const long long base = ptr[s] + lane;
    const int p0 = r >= 0 ? rowptr[r] : 0;
    for (int j = 0; j < (int)((ptr[s + 1] - ptr[s]) >> 5); ++j) {
        const long long d = base + 32LL * j;
        const bool in = j < len;
        scol[d] = in ? col[p0 + j] : 0;
        // a dense A's values: entry j of lane l at 32 VW (j / VW) + VW l + j % VW,
        // VW = 16 bytes / value size, so a lane reads VW entries per load
        const long long d64 = dense ? ptr[s] + 64LL * (j >> 1) + 2 * lane + (j & 1) : d;
        const long long d32 = dense ? ptr[s] + 128LL * (j >> 2) + 4 * lane + (j & 3) : d;
        if (sval) sval[d64] = in ? val[p0 + j] : 0.0;
        if (sval32) sval32[d32] = in ? val32[p0 + j] : 0.0f;
    }
}

// A dense A held as CSR: entry p = i*n + c has column c.
__global__ void k_dense_cols(int *__restrict__ col, long long nnz, int n) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz;
         p += (long long)gridDim.x * blockDim.x)
        col[p] = (int)(p % n);
}

void fill_dense_columns(rorbk_ctx *h) {
    const int g = std::max(1, std::min(8 * h->num_sms, (int)((h->nnz + 255) / 256)));
    k_dense_cols<<<g, 256, 0, h->stream>>>(h->col, h->nnz, (int)h->n);
}

// ------------------------------------------------- column-major copy of A
// Entries of column j in ascending rows.  Count per column, scan, place every
// entry at a free slot of its column (in any order), then order each column's
// slots by CSR position with rounds of pairwise merges of runs of 1, 2, 4, ...
// slots: a slot's place in the merged run is its index in its own run plus the
// number of slots of the other run that hold a smaller position (positions
// are distinct).  A row's entries are ascending in position, so the columns
// list their rows ascending.
__global__ void k_col_count(const int *__restrict__ col, long long nnz, int *__restrict__ cnt) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz;
         p += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[p]], 1);
}

__global__ void k_col_max(const int *__restrict__ cp, int n, int *__restrict__ out) {
    int v = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        v = max(v, cp[j + 1] - cp[j]);
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

__global__ void k_col_place(const int *__restrict__ rowptr, const int *__restrict__ col, int m,
                            const int *__restrict__ cp, int *__restrict__ fill, int *__restrict__ slot,
                            int *__restrict__ rowid) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            const int c = col[p];
            slot[cp[c] + atomicAdd(&fill[c], 1)] = p;
            rowid[p] = i;
        }
}

__global__ void k_col_merge(const int *__restrict__ col, const int *__restrict__ cp,
                            const int *__restrict__ in, int *__restrict__ out, long long nnz, int run) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz;
         q += (long long)gridDim.x * blockDim.x) {
        const int p = in[q];
        const int c = col[p];
        const long long s0 = cp[c];
        const int len = cp[c + 1] - (int)s0, o = (int)(q - s0);
        const int base = (int)(o / (2LL * run) * (2LL * run));
        const bool left = o - base < run;
        const int own0 = left ? base : base + run, oth0 = left ? base + run : base;
        const int othlen = max(0, min(run, len - oth0));
        const int *other = in + s0 + oth0;
        int lo = 0, hi = othlen;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (other[mid] < p) lo = mid + 1; else hi = mid;
        }
        out[s0 + base + (o - own0) + lo] = p;
    }
}

__global__ void k_col_gather(const int *__restrict__ slot, const int *__restrict__ rowid,
                             const double *__restrict__ val, const double *__restrict__ scale,
                             long long nnz, int *__restrict__ crow, double *__restrict__ cval,
                             float *__restrict__ cval32) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz;
         q += (long long)gridDim.x * blockDim.x) {
        const int p = slot[q], i = rowid[p];
        const double v = scale ? __ddiv_rn(val[p], scale[i]) : val[p];
        crow[q] = i;
        cval[q] = v;
        if (cval32) cval32[q] = __double2float_rn(v);
    }
}

// ---------------------------------------------------------------- driver
// Device scratch of one set-up pass, freed when the pass ends (after the
// stream has drained).
struct Scratch {
    cudaStream_t s;
    std::vector<void *> p;
    explicit Scratch(cudaStream_t s_) : s(s_) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    template <typename T>
    T *get(size_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return (T *)q;
    }
    ~Scratch() {
        if (p.empty()) return;
        cudaStreamSynchronize(s);
        for (void *q : p) cudaFree(q);
    }
};

// A buffer the handle keeps: allocated on the first set-up pass, reused by a
// refresh of the values (same pattern, same size).
template <typename T>
static bool keep(rorbk_ctx *h, T *&ptr, size_t count) {
    if (!ptr) ptr = (T *)dev_alloc(h, std::max<size_t>(count, 1) * sizeof(T));
    return ptr != nullptr;
}

// Exclusive scan of n ints in place; *grand_total_host receives the sum.
static rorbk_status scan_device(rorbk_ctx *h, int *d, long long n, int *grand_total_host) {
    const int nt = 256;
    long long tiles = (n + nt - 1) / nt;
    Scratch sc(h->stream);
    int *sums = sc.get<int>(tiles + 1);
    int *tot = sc.get<int>(1);
    if (!sums || !tot) return fail(h, RORBK_ERR_OOM, "scan workspace");
    k_scan_tiles<<<(unsigned)tiles, nt, 0, h->stream>>>(d, d, sums, n);
    k_scan_sums<<<1, 1024, 0, h->stream>>>(sums, (int)tiles, tot);
    k_scan_add<<<(unsigned)tiles, nt, 0, h->stream>>>(d, sums, n);
    rorbk_status st = cuda_check(h, cudaMemcpyAsync(grand_total_host, tot, sizeof(int),
                                                    cudaMemcpyDeviceToHost, h->stream), "scan total");
    if (st) return st;
    return cuda_check(h, cudaStreamSynchronize(h->stream), "scan");
}

// Rows sorted by length (longest first, ties by row) into slices of 32.  On a
// refresh of the values only the values are copied again.
static rorbk_status build_sell(rorbk_ctx *h, const std::vector<int> &hrp, bool refresh) {
    auto &S = h->sell;
    cudaStream_t st = h->stream;
    if (!refresh) {
        const int m = (int)h->m;
        int maxlen = 0;
        for (int i = 0; i < m; ++i) maxlen = std::max(maxlen, hrp[i + 1] - hrp[i]);
        std::vector<int> cnt(maxlen + 2, 0);
        for (int i = 0; i < m; ++i) cnt[hrp[i + 1] - hrp[i]]++;
        std::vector<int> start(maxlen + 2, 0);      // descending length order
        for (int L = maxlen, acc = 0; L >= 0; --L) { start[L] = acc; acc += cnt[L]; }
        std::vector<int> order(m);
        for (int i = 0; i < m; ++i) order[start[hrp[i + 1] - hrp[i]]++] = i;
        const int ns = (m + 31) / 32;
        std::vector<long long> ptr(ns + 1, 0);
        std::vector<int> len(ns), row((size_t)ns * 32, -1), rlen((size_t)ns * 32, 0);
        for (int sl = 0; sl < ns; ++sl) {
            int L = 0;
            for (int l = 0; l < 32; ++l) {
                const int q = sl * 32 + l;
                if (q < m) {
                    row[q] = order[q];
                    rlen[q] = hrp[order[q] + 1] - hrp[order[q]];
                    L = std::max(L, rlen[q]);
                }
            }
            len[sl] = L;
            // a dense A's slices span a multiple of 4 entries per lane (its values
            // are grouped 4 (FP32) or 2 (FP64) entries per lane)
            const int Lp = h->format == RORBK_FORMAT_DENSE ? (L + 3) & ~3 : L;
            ptr[sl + 1] = ptr[sl] + 32LL * Lp;
        }
        S.nslices = ns;
        S.ptr = (long long *)dev_alloc(h, (ns + 1) * sizeof(long long));
        S.len = (int *)dev_alloc(h, ns * sizeof(int));
        S.row = (int *)dev_alloc(h, (size_t)ns * 32 * sizeof(int));
        S.rlen = (int *)dev_alloc(h, (size_t)ns * 32 * sizeof(int));
        const long long ent = std::max(1LL, ptr[ns]);
        S.col = (int *)dev_alloc(h, ent * sizeof(int));
        if (h->vdtype == RORBK_F64) S.val = (double *)dev_alloc(h, ent * sizeof(double));
        if (h->val32) S.val32 = (float *)dev_alloc(h, ent * sizeof(float));
        if (!S.ptr || !S.len || !S.row || !S.rlen || !S.col || (h->vdtype == RORBK_F64 && !S.val) ||
            (h->val32 && !S.val32))
            return fail(h, RORBK_ERR_OOM, "SELL copy of A");
        cudaMemcpyAsync(S.ptr, ptr.data(), (ns + 1) * sizeof(long long), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(S.len, len.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(S.row, row.data(), (size_t)ns * 32 * sizeof(int), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(S.rlen, rlen.data(), (size_t)ns * 32 * sizeof(int), cudaMemcpyHostToDevice, st);
    }
    const int ns = S.nslices;
    k_sell_fill<<<(unsigned)((ns * 32LL + 255) / 256), 256, 0, st>>>(
        h->rowptr, h->col, h->val, h->val32, ns, S.ptr, S.row, S.rlen, S.col, S.val, S.val32,
        h->format == RORBK_FORMAT_DENSE ? 1 : 0);
    return cuda_check(h, cudaStreamSynchronize(st), "SELL copy of A");
}

// Local rows of every block ordered by length, longest first (ties by row):
// the static update gives one row per thread, and a warp's fused
// multiply-add chain is as long as its longest row.
static rorbk_status build_block_order(rorbk_ctx *h, const std::vector<int> &hrp) {
    const int k = h->k;
    std::vector<uint16_t> perm(h->m);
    std::vector<int> idx;
    for (int t = 0; t < k; ++t) {
        const int r0 = (int)h->h_off[t], s = (int)(h->h_off[t + 1] - h->h_off[t]);
        idx.resize(s);
        for (int a = 0; a < s; ++a) idx[a] = a;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            return hrp[r0 + x + 1] - hrp[r0 + x] > hrp[r0 + y + 1] - hrp[r0 + y];
        });
        for (int a = 0; a < s; ++a) perm[r0 + a] = (uint16_t)idx[a];
    }
    h->ops.bperm = (uint16_t *)dev_alloc(h, (size_t)h->m * sizeof(uint16_t));
    if (!h->ops.bperm) return fail(h, RORBK_ERR_OOM, "block row order");
    return cuda_check(h, cudaMemcpyAsync(h->ops.bperm, perm.data(), (size_t)h->m * sizeof(uint16_t),
                                         cudaMemcpyHostToDevice, h->stream), "block row order");
}

// Everything of Algorithm 1's set-up that follows from A: validation, the
// SELL copy, row norms, block transposes and coupled rows, centroids, C and
// the proposal, and the static operators.  With refresh (new values, same
// pattern) every buffer is reused and only the value-dependent parts are
// formed again, by the same kernels in the same order, so the result equals a
// fresh set-up bit for bit.
rorbk_status build_setup(rorbk_ctx *h, const std::vector<int> &hrp, bool refresh) {
    cudaStream_t s = h->stream;
    const int m = (int)h->m, n = (int)h->n, k = h->k;
    rorbk_status st;
    Scratch sc(s);
    int *flags = sc.get<int>(2);
    if (!flags) return fail(h, RORBK_ERR_OOM, "flags");
    cudaMemsetAsync(flags, 0, 2 * sizeof(int), s);
    int gs = std::max(1, std::min(4 * h->num_sms, (m + 255) / 256));
    k_validate_csr<<<gs, 256, 0, s>>>(h->rowptr, h->col, h->val, m, n, flags);
    int hf[2] = {0, 0};
    if ((st = cuda_check(h, cudaMemcpyAsync(hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s), "validate")))
        return st;
    if ((st = cuda_check(h, cudaStreamSynchronize(s), "validate"))) return st;
    if (hf[0] & 1)
        return fail(h, RORBK_ERR_INVALID_ARG,
                    "CSR structure: row_ptr must be non-decreasing and columns strictly ascending in [0,n)");
    if (hf[0] & 2) return fail(h, RORBK_ERR_NUMERIC, "A holds NaN or Inf");
    if (!keep(h, h->blk_nz, k + 1)) return fail(h, RORBK_ERR_OOM, "block entry offsets");
    k_block_nz<<<std::max(1, (k + 256) / 256), 256, 0, s>>>(h->rowptr, h->off, k, h->blk_nz);
    if ((st = build_sell(h, hrp, refresh))) return st;
    if (!refresh && (st = build_block_order(h, hrp))) return st;
    // row norms for the dynamic update: from the FP64 values, and from the
    // FP32 copy that the mixed form's inner solve reads when it differs
    if (!keep(h, h->rn, m)) return fail(h, RORBK_ERR_OOM, "row norms");
    k_row_norms<double><<<gs, 256, 0, s>>>(h->rowptr, h->val, m, h->rn);
    if (!refresh) h->rn32 = h->rn;
    if (h->val32 && h->vdtype == RORBK_F64) {
        if (h->rn32 == h->rn) h->rn32 = nullptr;
        if (!keep(h, h->rn32, m)) return fail(h, RORBK_ERR_OOM, "row norms");
        k_row_norms<float><<<gs, 256, 0, s>>>(h->rowptr, h->val32, m, h->rn32);
    }

    // block transpose, coupled rows
    const long long nnz = h->nnz;
    unsigned char *coupled = sc.get<unsigned char>(m);
    int *ncoupled = sc.get<int>(k + 1);
    if (!keep(h, h->bt.col, nnz + 16) || !keep(h, h->bt.row, nnz + 16) || !keep(h, h->bt.val, nnz + 16) ||
        !keep(h, h->bt.off16, nnz + 16) ||
        !keep(h, h->bt.seg, nnz) || !keep(h, h->bt.seg_ptr, k) || !coupled || !ncoupled)
        return fail(h, RORBK_ERR_OOM, "block transpose");
    if (h->format == RORBK_FORMAT_DENSE) {
        const int gx = std::max(1, std::min(4 * h->num_sms, (int)((h->nnz / k + 255) / 256)));
        k_block_transpose_dense<<<dim3(gx, k), 256, 0, s>>>(h->val, h->off, n, h->bt.col, h->bt.row, h->bt.val,
                                                            h->bt.off16, h->bt.seg, h->bt.seg_ptr, coupled,
                                                            ncoupled);
    } else {
        k_block_transpose<<<k, 256, 0, s>>>(h->rowptr, h->col, h->val, h->off, h->bt.col, h->bt.row,
                                            h->bt.val, h->bt.off16, h->bt.seg, h->bt.seg_ptr, coupled, ncoupled);
    }
    if ((st = cuda_check(h, cudaGetLastError(), "block transpose"))) return st;

    // centroids, C row sums, proposal
    {
        Scratch cs(s);
        int *colcnt = cs.get<int>(n + 1);
        int *fill = cs.get<int>(n + 1);
        if (!colcnt || !fill) return fail(h, RORBK_ERR_OOM, "centroid columns");
        cudaMemsetAsync(colcnt, 0, (size_t)(n + 1) * sizeof(int), s);
        cudaMemsetAsync(fill, 0, (size_t)(n + 1) * sizeof(int), s);
        int gk = std::min(k, 8 * h->num_sms);
        k_centroid_count<<<gk, 128, 0, s>>>(h->rowptr, h->off, h->bt.col, h->bt.seg, h->bt.seg_ptr,
                                           k, colcnt);
        int total = 0;
        if ((st = scan_device(h, colcnt, (long long)n + 1, &total))) return st;
        int *cb = cs.get<int>(std::max(1, total));
        double *cv = cs.get<double>(std::max(1, total));
        double *G = cs.get<double>((size_t)k * k);
        if (!cb || !cv || !G) return fail(h, RORBK_ERR_OOM, "centroid Gram");
        k_centroid_fill<<<gk, 128, 0, s>>>(h->rowptr, h->off, h->bt.col, h->bt.val, h->bt.seg,
                                          h->bt.seg_ptr, k, colcnt, fill, cb, cv);
        cudaMemsetAsync(G, 0, (size_t)k * k * sizeof(double), s);
        k_centroid_gram<<<(k * 32 + 255) / 256, 256, 0, s>>>(h->rowptr, h->off, h->bt.col, h->bt.val,
                                                            h->bt.seg, h->bt.seg_ptr, k, colcnt,
                                                            cb, cv, G);
        k_crowsum<<<(k * 32 + 255) / 256, 256, 0, s>>>(G, k, h->crowsum);
        k_proposal<<<1, 1024, 0, s>>>(h->crowsum, k, (double)n, h->cdf, h->pbar);
        if ((st = cuda_check(h, cudaGetLastError(), "proposal"))) return st;
    }

    // static operators on the coupled rows of every block
    {
        std::vector<int> hcnt(k + 1, 0);
        if ((st = cuda_check(h, cudaMemcpyAsync(hcnt.data(), ncoupled, k * sizeof(int),
                                                cudaMemcpyDeviceToHost, s), "coupled counts")))
            return st;
        if ((st = cuda_check(h, cudaStreamSynchronize(s), "coupled counts"))) return st;
        // blocks with at least n rows take the n x n form (Lemma 1, Section 3.1)
        std::vector<long long> woodp(k, -1);
        long long wtot = 0;
        h->n_wood = 0;
        for (int t = 0; t < k; ++t)
            if (h->h_off[t + 1] - h->h_off[t] >= n) {
                woodp[t] = wtot;
                wtot += (long long)n * n;
                hcnt[t] = 0;
                ++h->n_wood;
            }
        if (h->n_wood) {
            if (!keep(h, h->wood_ptr, k) || !keep(h, h->wood_ss, wtot))
                return fail(h, RORBK_ERR_OOM, "s >= n operators");
            cudaMemcpyAsync(h->wood_ptr, woodp.data(), (size_t)k * sizeof(long long), cudaMemcpyHostToDevice, s);
        }
        std::vector<int> sptr(k + 1, 0);
        std::vector<long long> wptr(k + 1, 0);
        for (int t = 0; t < k; ++t) {
            sptr[t + 1] = sptr[t] + hcnt[t];
            wptr[t + 1] = wptr[t] + (long long)hcnt[t] * hcnt[t];
        }
        if (!keep(h, h->ops.s_ptr, k + 1) || !keep(h, h->ops.w_ptr, k + 1) ||
            !keep(h, h->ops.s_idx, std::max(1, sptr[k])) || !keep(h, h->ops.s_pos, m) ||
            !keep(h, h->ops.w_ss, std::max(1LL, wptr[k])) || !keep(h, h->ops.w_diag, m))
            return fail(h, RORBK_ERR_OOM, "static operators");
        double *linv = sc.get<double>(std::max(1LL, wptr[k]));
        if (!linv) return fail(h, RORBK_ERR_OOM, "static operator scratch");
        cudaMemcpyAsync(h->ops.s_ptr, sptr.data(), (k + 1) * sizeof(int), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(h->ops.w_ptr, wptr.data(), (k + 1) * sizeof(long long), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(flags, 0, sizeof(int), s);
        // a dense A: every block's Gram by the grid (the blocks' rows are long)
        const bool dense_gram = h->format == RORBK_FORMAT_DENSE && !h->n_wood;
        if (dense_gram) {
            const int nt = (h->smax + kSgT - 1) / kSgT;
            k_dense_static_gram<<<dim3(nt * (nt + 1) / 2, k), kSgT * kSgT, 0, s>>>(h->val, h->off, n, h->mu,
                                                                                 h->ops.w_ptr, h->ops.w_ss);
        }
        k_static_ops<<<k, 256, 0, s>>>(h->rowptr, h->col, h->val, h->off, h->mu, coupled,
                                       h->ops.s_ptr, h->ops.w_ptr, h->ops.s_idx, h->ops.s_pos,
                                       h->ops.w_ss, h->ops.w_diag, linv, h->wood_ptr, flags,
                                       dense_gram ? 1 : 0);
        if (h->n_wood) {
            double *linv2 = sc.get<double>(wtot);
            if (!linv2) return fail(h, RORBK_ERR_OOM, "s >= n operator scratch");
            k_wood_ops<<<k, 256, 0, s>>>(h->rowptr, h->off, (int)n, h->mu, h->wood_ptr, h->bt.col, h->bt.row,
                                         h->bt.val, h->wood_ss, linv2, flags);
        }
        int spd = 0;
        st = cuda_check(h, cudaMemcpyAsync(&spd, flags, sizeof(int), cudaMemcpyDeviceToHost, s), "static ops");
        if (!st) st = cuda_check(h, cudaStreamSynchronize(s), "static ops");
        if (st) return st;
        if (spd) return fail(h, RORBK_ERR_NOT_SPD, "a static block Gram is not positive definite (lambda = 0 with dependent rows?)");
        if (h->precision_built) {
            if (!keep(h, h->ops.w_ss32, std::max(1LL, wptr[k])) || !keep(h, h->ops.w_diag32, m) ||
                !keep(h, h->bt.val32, nnz + 16))
                return fail(h, RORBK_ERR_OOM, "fp32 operators");
            k_narrow<<<gs, 256, 0, s>>>(h->ops.w_ss, h->ops.w_ss32, std::max(1LL, wptr[k]));
            k_narrow<<<gs, 256, 0, s>>>(h->ops.w_diag, h->ops.w_diag32, m);
            k_narrow<<<gs, 256, 0, s>>>(h->bt.val, h->bt.val32, nnz);
            if (h->n_wood) {
                if (!keep(h, h->wood_ss32, wtot)) return fail(h, RORBK_ERR_OOM, "fp32 s >= n operators");
                k_narrow<<<gs, 256, 0, s>>>(h->wood_ss, h->wood_ss32, wtot);
            }
        }
    }
    return cuda_check(h, cudaStreamSynchronize(s), "setup");
}

rorbk_status build_csc(rorbk_ctx *h, const double *scale, int *cp, int *crow, double *cval, float *cval32) {
    cudaStream_t s = h->stream;
    const int m = (int)h->m, n = (int)h->n;
    const long long nnz = h->nnz;
    rorbk_status st;
    Scratch sc(s);
    int *fill = sc.get<int>(n);
    int *slot = sc.get<int>(nnz), *slot2 = sc.get<int>(nnz), *rowid = sc.get<int>(nnz);
    int *maxlen = sc.get<int>(1);
    if (!fill || !slot || !slot2 || !rowid || !maxlen) return fail(h, RORBK_ERR_OOM, "column-major copy of A");
    const int ge = (int)std::max(1LL, std::min<long long>(8LL * h->num_sms, (nnz + 255) / 256));
    const int gr = std::max(1, std::min(8 * h->num_sms, (m + 255) / 256));
    cudaMemsetAsync(cp, 0, (size_t)(n + 1) * sizeof(int), s);
    cudaMemsetAsync(fill, 0, (size_t)n * sizeof(int), s);
    cudaMemsetAsync(maxlen, 0, sizeof(int), s);
    k_col_count<<<ge, 256, 0, s>>>(h->col, nnz, cp);
    int total = 0;
    if ((st = scan_device(h, cp, (long long)n + 1, &total))) return st;
    if (total != nnz) return fail(h, RORBK_ERR_CUDA, "column-major copy of A: entry count");
    k_col_max<<<std::max(1, std::min(8 * h->num_sms, (n + 255) / 256)), 256, 0, s>>>(cp, n, maxlen);
    k_col_place<<<gr, 256, 0, s>>>(h->rowptr, h->col, m, cp, fill, slot, rowid);
    int L = 0;
    if ((st = cuda_check(h, cudaMemcpyAsync(&L, maxlen, sizeof(int), cudaMemcpyDeviceToHost, s), "column lengths")))
        return st;
    if ((st = cuda_check(h, cudaStreamSynchronize(s), "column lengths"))) return st;
    for (int run = 1; run < L; run *= 2) {
        k_col_merge<<<ge, 256, 0, s>>>(h->col, cp, slot, slot2, nnz, run);
        std::swap(slot, slot2);
    }
    k_col_gather<<<ge, 256, 0, s>>>(slot, rowid, h->val, scale, nnz, crow, cval, cval32);
    return cuda_check(h, cudaStreamSynchronize(s), "column-major copy of A");
}

}  // namespace rorbk
