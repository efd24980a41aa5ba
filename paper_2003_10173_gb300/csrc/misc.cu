// Small helper kernels of the construction phase: counter-based Gaussian
// probes, row gathers/scatters between the caller's node order and tree order,
// finiteness scans and list sums of small matrices.
#include "common.h"

namespace h2 {

namespace {

constexpr int NT = 256;

// Gaussian of entry (row, col) by Box-Muller from two SplitMix64 outputs.
__device__ inline double gauss_at(uint64_t key, uint64_t row, uint64_t col) {
    const uint64_t c = (col << 32) + row;
    const uint64_t b1 = splitmix_at(key, 2ull * c);
    const uint64_t b2 = splitmix_at(key, 2ull * c + 1ull);
    const double u1 = (double)((b1 >> 11) + 1ull) * 0x1p-53;
    const double u2 = (double)(b2 >> 11) * 0x1p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

__global__ void fill_zero_kernel(double* p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

__global__ void probe_fill_kernel(int64_t N, int ncols, int col0, const int32_t* __restrict__ perm,
                                  const int32_t* __restrict__ row_box, int shift, uint64_t key,
                                  double* __restrict__ Om, double* __restrict__ Omt) {
    const int64_t total = N * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N;
        const int j = (int)(e / N);
        const int box = row_box[i] >> shift;
        double v = 0.0;
        if ((box & 1) == 0) v = gauss_at(key, (uint64_t)i, (uint64_t)(col0 + j));
        Om[perm[i] + (int64_t)j * N] = v;
        if (Omt) Omt[i + (int64_t)j * N] = v;
    }
}

// Coloured probes: column block c (q columns) is Gaussian on the rows whose level box has colour c.
__global__ void probe_colored_kernel(int64_t N, int q, int ncols, const int32_t* __restrict__ perm,
                                     const int32_t* __restrict__ row_box, int shift,
                                     const int32_t* __restrict__ color, uint64_t key, double* __restrict__ Om,
                                     double* __restrict__ Omt) {
    const int64_t total = N * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N;
        const int j = (int)(e / N);
        const int c = color[row_box[i] >> shift];
        const double v = (c >= 0 && j / q == c) ? gauss_at(key, (uint64_t)i, (uint64_t)j) : 0.0;
        Om[perm[i] + (int64_t)j * N] = v;
        if (Omt) Omt[i + (int64_t)j * N] = v;
    }
}

__global__ void gaussian_vector_kernel(int64_t N, const int32_t* __restrict__ perm, uint64_t key,
                                       double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        x[perm[i]] = gauss_at(key, (uint64_t)i, 0ull);
}

__global__ void gather_kernel(int64_t N, int ncols, const int32_t* __restrict__ perm,
                              const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                              int64_t ldd) {
    const int64_t total = N * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, j = e / N;
        dst[i + j * ldd] = src[perm[i] + j * lds];
    }
}

__global__ void scatter_kernel(int64_t N, int ncols, const int32_t* __restrict__ perm,
                               const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                               int64_t ldd) {
    const int64_t total = N * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, j = e / N;
        dst[perm[i] + j * ldd] = src[i + j * lds];
    }
}

__global__ void scan_finite_kernel(int64_t N, int ncols, const double* __restrict__ x, int64_t ld,
                                   int* __restrict__ flag) {
    const int64_t total = N * ncols;
    bool bad = false;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, j = e / N;
        if (!isfinite(x[i + j * ld])) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

__global__ void sum_lists_kernel(const int64_t* __restrict__ out_off, const int* __restrict__ len,
                                 const int* __restrict__ beg, const int* __restrict__ end,
                                 const int64_t* __restrict__ in_off, const double* __restrict__ in,
                                 double* __restrict__ out, int accumulate) {
    const int o = blockIdx.x;
    const int n = len[o];
    const int b = beg[o], en = end[o];
    double* dst = out + out_off[o];
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        double s = accumulate ? dst[e] : 0.0;
        for (int j = b; j < en; ++j) s += in[in_off[j] + e];
        dst[e] = s;
    }
}

__global__ void col_sqnorms_kernel(int64_t N, const double* __restrict__ x, int64_t ld, double* __restrict__ out) {
    const double* c = x + blockIdx.x * ld;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s = fma(c[i], c[i], s);
    __shared__ double sh[NT / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += sh[w];
        out[blockIdx.x] = t;
    }
}

__global__ void scale_cols_kernel(int64_t N, int ncols, double* __restrict__ x, int64_t ld,
                                  const double* __restrict__ sc) {
    const int64_t total = N * ncols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, j = e / N;
        x[i + j * ld] *= sc[j];
    }
}

__global__ void block_op_kernel(int kind, const BlkDesc* __restrict__ desc, const double* __restrict__ src,
                                double* __restrict__ dst) {
    const BlkDesc d = desc[blockIdx.x];
    const int n = d.rows * d.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int i = e % d.rows, j = e / d.rows;
        double v;
        if (kind == BLK_IDENTITY) v = (i == j) ? 1.0 : 0.0;
        else if (kind == BLK_COPY) v = src[d.src_off + i + (int64_t)j * d.lds];
        else v = 0.5 * (src[d.src_off + i + (int64_t)j * d.lds] + src[d.src_off + j + (int64_t)i * d.lds]);
        dst[d.dst_off + i + (int64_t)j * d.ldd] = v;
    }
}

inline unsigned grid_for(int64_t total) {
    int64_t b = (total + NT - 1) / NT;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

uint64_t rng_key(uint64_t seed, int stream_id, int level) {
    return mix64(seed ^ mix64(((uint64_t)stream_id << 16) + (uint64_t)level));
}

void fill_zero(double* p, size_t count, cudaStream_t s) {
    if (!count) return;
    fill_zero_kernel<<<grid_for((int64_t)count), NT, 0, s>>>(p, count);
    after_launch("fill_zero");
}

void probe_fill(int64_t N, int ncols, int col0, const int32_t* d_perm, const int32_t* d_row_box,
                int level_shift, uint64_t seed, int stream_id, int level, double* Om_orig,
                double* Om_tree, cudaStream_t s) {
    if (N * ncols == 0) return;
    probe_fill_kernel<<<grid_for(N * ncols), NT, 0, s>>>(N, ncols, col0, d_perm, d_row_box, level_shift,
                                                          rng_key(seed, stream_id, level), Om_orig, Om_tree);
    after_launch("probe_fill");
}

void probe_fill_colored(int64_t N, int q, int ncolors, const int32_t* d_perm, const int32_t* d_row_box,
                        int level_shift, const int32_t* d_color, uint64_t seed, int stream_id, int level,
                        double* Om_orig, double* Om_tree, cudaStream_t s) {
    const int ncols = q * ncolors;
    if (N * ncols == 0) return;
    probe_colored_kernel<<<grid_for(N * ncols), NT, 0, s>>>(N, q, ncols, d_perm, d_row_box, level_shift, d_color,
                                                             rng_key(seed, stream_id, level), Om_orig, Om_tree);
    after_launch("probe_colored");
}

void gaussian_vector(int64_t N, const int32_t* d_perm, uint64_t seed, int stream_id, double* x_orig,
                     cudaStream_t s) {
    gaussian_vector_kernel<<<grid_for(N), NT, 0, s>>>(N, d_perm, rng_key(seed, stream_id, 0), x_orig);
    after_launch("gaussian_vector");
}

void gather_rows(int64_t N, int ncols, const int32_t* d_perm, const double* src, int64_t lds,
                 double* dst, int64_t ldd, cudaStream_t s) {
    if (N * ncols == 0) return;
    gather_kernel<<<grid_for(N * ncols), NT, 0, s>>>(N, ncols, d_perm, src, lds, dst, ldd);
    after_launch("gather_rows");
}

void scatter_rows(int64_t N, int ncols, const int32_t* d_perm, const double* src, int64_t lds,
                  double* dst, int64_t ldd, cudaStream_t s) {
    if (N * ncols == 0) return;
    scatter_kernel<<<grid_for(N * ncols), NT, 0, s>>>(N, ncols, d_perm, src, lds, dst, ldd);
    after_launch("scatter_rows");
}

void scan_finite(int64_t N, int ncols, const double* x, int64_t ld, int* d_flag, cudaStream_t s) {
    if (N * ncols == 0) return;
    scan_finite_kernel<<<grid_for(N * ncols), NT, 0, s>>>(N, ncols, x, ld, d_flag);
    after_launch("scan_finite");
}


void sum_lists(int count, const int64_t* d_out_off, const int* d_len, const int* d_begin,
               const int* d_end, const int64_t* d_in_off, const double* in, double* out,
               int accumulate, cudaStream_t s) {
    if (count <= 0) return;
    sum_lists_kernel<<<count, NT, 0, s>>>(d_out_off, d_len, d_begin, d_end, d_in_off, in, out, accumulate);
    after_launch("sum_lists");
}

void col_sqnorms(int64_t N, int ncols, const double* x, int64_t ld, double* out, cudaStream_t s) {
    if (ncols <= 0) return;
    col_sqnorms_kernel<<<ncols, NT, 0, s>>>(N, x, ld, out);
    after_launch("col_sqnorms");
}

void block_op(int kind, int count, const BlkDesc* d_desc, const double* src, double* dst, cudaStream_t s) {
    if (count <= 0) return;
    block_op_kernel<<<count, NT, 0, s>>>(kind, d_desc, src, dst);
    after_launch("block_op");
}

void scale_cols(int64_t N, int ncols, double* x, int64_t ld, const double* d_scale, cudaStream_t s) {
    if (N * ncols == 0) return;
    scale_cols_kernel<<<grid_for(N * ncols), NT, 0, s>>>(N, ncols, x, ld, d_scale);
    after_launch("scale_cols");
}

}  // namespace h2
