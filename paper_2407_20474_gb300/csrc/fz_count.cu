// fz_count.cu -- the exact counting table of the factorization sets.
//
//   C[j][r] = |Z(r, (g_{j+1}, ..., g_d))|,  j = 0..d (0-based), r = 0..n,
//   C[d][r] = [r == 0],   C[j][r] = sum_{t >= 0} C[j+1][r - t g_{j+1}].
//
// By the disjoint recurrence of Section 2 (Lemma "disjdyn") C[i-1][r] is
// |Z_{>=i}(r)|, the size of the block incr_i(Z_{>=i}(r)) = Z_{=i}(r + g_i)
// whose saving the paper describes in Section 2.3.  It gives every block's
// size and start, hence exact output offsets for every warp.
//
// Each row is a strided inclusive prefix sum of the row below it (stride
// g_{j+1}): for every residue class rho mod g the entries rho, rho + g, ...
// are summed in order.  Short chains are scanned by one warp each; long
// chains are cut into blocks of RB entries, the block sums are scanned by the
// same routine (they form a strided array of the same shape), and the blocks
// are then re-walked with their carries.  All sums saturate at 2^64 - 1.
#include <cstdlib>
#include <cstring>

#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int64_t DIRECT_T = 4096;  // chains up to this length: one warp each
constexpr int64_t LANE_T = 1024;    // chains up to this length, 32 or more: one lane each
constexpr int LANE_ILP = 8;
constexpr int RB = 32;              // entries per block in the blocked scan
constexpr int THREADS = 256;

__global__ void row_delta_kernel(uint64_t *__restrict__ row, int64_t len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < len; i += stride) row[i] = (i == 0) ? 1ull : 0ull;
}

// One warp per residue chain; 4 x 32 entries loaded ahead of the scan.
__global__ void __launch_bounds__(THREADS)
chain_scan_direct_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                         int64_t len, int64_t g) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t chains = g < len ? g : len;
    for (int64_t rho = warp; rho < chains; rho += nwarps) {
        const int64_t T = (len - rho + g - 1) / g;
        uint64_t carry = 0;
        for (int64_t t0 = 0; t0 < T; t0 += 128) {
            uint64_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t t = t0 + u * 32 + lane;
                v[u] = t < T ? __ldg(in + rho + t * g) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t t = t0 + u * 32 + lane;
                uint64_t s = sat_add(warp_incl_scan_sat(v[u], lane), carry);
                if (t < T) out[rho + t * g] = s;
                carry = shfl_u64(s, 31);
            }
        }
    }
}

// S[b*g + rho] = sum of the RB entries of chain rho in block b.
__global__ void __launch_bounds__(THREADS)
block_sum_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ S, int64_t len,
                 int64_t g, int64_t slen) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < slen; i += stride) {
        const int64_t b = i / g, rho = i - b * g;
        const int64_t r0 = (b * RB) * g + rho;
        uint64_t acc = 0;
#pragma unroll 8
        for (int t = 0; t < RB; ++t) {
            int64_t r = r0 + (int64_t)t * g;
            if (r < len) acc = sat_add(acc, __ldg(in + r));
        }
        S[i] = acc;
    }
}

// out[r] = carry(block) + running sum inside the block.  At most 64
// registers (4 blocks per SM), so that it fits beside an enumeration capped
// at 3 blocks per SM.
__global__ void __launch_bounds__(THREADS, 4)
block_apply_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                   const uint64_t *__restrict__ Sincl, int64_t len, int64_t g, int64_t slen) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < slen; i += stride) {
        const int64_t b = i / g, rho = i - b * g;
        uint64_t acc = b > 0 ? Sincl[i - g] : 0ull;
        const int64_t r0 = (b * RB) * g + rho;
#pragma unroll 4
        for (int t = 0; t < RB; ++t) {
            int64_t r = r0 + (int64_t)t * g;
            if (r < len) {
                acc = sat_add(acc, __ldg(in + r));
                out[r] = acc;
            }
        }
    }
}

int grid_for(int64_t work, int per_block) {
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

// Scratch words the blocked scan needs for an array of `len` entries, stride g.
int64_t scan_tmp_words(int64_t len, int64_t g) {
    int64_t T = (len + g - 1) / g;
    if (len <= 0 || T <= DIRECT_T) return 0;
    int64_t nrb = (T + RB - 1) / RB;
    int64_t slen = nrb * g;
    return 2 * slen + scan_tmp_words(slen, g);
}

// out[r] = sum_{t >= 0, r - t g >= 0} in[r - t g], for r < len.
int strided_scan(const uint64_t *in, uint64_t *out, int64_t len, int64_t g, uint64_t *tmp,
                 cudaStream_t s) {
    if (len <= 0) return FZ_OK;
    const int64_t T = (len + g - 1) / g;
    if (T <= DIRECT_T) {
        int64_t chains = g < len ? g : len;
        int blocks = grid_for(chains * 32, THREADS);
        chain_scan_direct_kernel<<<blocks, THREADS, 0, s>>>(in, out, len, g);
        note_launch();
        FZ_CUDA_TRY(cudaGetLastError());
        return FZ_OK;
    }
    const int64_t nrb = (T + RB - 1) / RB;
    const int64_t slen = nrb * g;
    uint64_t *S = tmp, *Sincl = tmp + slen;
    block_sum_kernel<<<grid_for(slen, THREADS), THREADS, 0, s>>>(in, S, len, g, slen);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    int rc = strided_scan(S, Sincl, slen, g, tmp + 2 * slen, s);
    if (rc != FZ_OK) return rc;
    block_apply_kernel<<<grid_for(slen, THREADS), THREADS, 0, s>>>(in, out, Sincl, len, g, slen);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

}  // namespace

int64_t count_table_tmp_words(const int32_t *g, int d, int32_t n) {
    int64_t w = 0;
    for (int j = 0; j < d; ++j) {
        int64_t t = scan_tmp_words((int64_t)n + 1, g[j]);
        if (t > w) w = t;
    }
    return w;
}

int64_t exclusive_scan_tmp_words(int64_t len) { return scan_tmp_words(len, 1); }

int launch_count_table_tmp(const int32_t *g, int d, int32_t n, uint64_t *table, uint64_t *tmp,
                           cudaStream_t s) {
    const int64_t len = (int64_t)n + 1;
    uint64_t *last = table + (int64_t)d * len;
    row_delta_kernel<<<grid_for(len, THREADS), THREADS, 0, s>>>(last, len);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    for (int j = d - 1; j >= 0; --j) {
        int rc = strided_scan(table + (int64_t)(j + 1) * len, table + (int64_t)j * len, len,
                              g[j], tmp, s);
        if (rc != FZ_OK) return rc;
    }
    return FZ_OK;
}

__global__ void row_ones_kernel(uint64_t *__restrict__ row, int64_t len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < len; i += stride) row[i] = 1ull;
}

// Number of depth-lam nodes (runs of sibling leaves) under a node at depth j
// with remainder x: RT[lam][x] = 1 and RT[j] = RT[j+1] strided-summed with
// stride g_j -- the count-table recurrence over the leading generators.
int launch_runs_table(const int32_t *g, int lam, int32_t n, uint64_t *RT, uint64_t *tmp,
                      int clamp_row, int64_t clamp_top, cudaStream_t s) {
    const int64_t len = (int64_t)n + 1;
    row_ones_kernel<<<grid_for(len, THREADS), THREADS, 0, s>>>(RT + (int64_t)lam * len, len);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    for (int j = lam - 1; j >= 0; --j) {
        int rc = strided_scan(RT + (int64_t)(j + 1) * len, RT + (int64_t)j * len, len, g[j],
                              tmp, s);
        if (rc != FZ_OK) return rc;
        if (j == clamp_row && clamp_top > 0) {
            const int64_t m = clamp_top < len ? clamp_top : len;
            row_ones_kernel<<<grid_for(m, THREADS), THREADS, 0, s>>>(RT + (int64_t)j * len, m);
            note_launch();
            FZ_CUDA_TRY(cudaGetLastError());
        }
    }
    return FZ_OK;
}

// ---------------------------------------------------------------------------
// Batched strided scans: many independent rows (of many instances' count and
// runs tables) in one launch.  Each CTA executes one task: a range of chains
// scanned directly (one warp per chain), a range of block sums, a range of
// chains of block sums, a range of block applications, or a range of a row
// initialisation (delta or ones).
// ---------------------------------------------------------------------------
// Logical entry r of a job's rows is entry off + r * es of the table row
// (es = 1, off = 0: the whole row; es = g_1, off = n mod g_1: the one chain
// of row 0 that is ever read).
__device__ __forceinline__ void chain_scan_warp(const uint64_t *__restrict__ in,
                                                uint64_t *__restrict__ out, int64_t len,
                                                int64_t g, int64_t rho, int lane,
                                                int64_t ones_below = 0, int64_t off = 0,
                                                int64_t es = 1) {
    const int64_t T = (len - rho + g - 1) / g;
    uint64_t carry = 0;
    for (int64_t t0 = 0; t0 < T; t0 += 128) {
        uint64_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int64_t t = t0 + u * 32 + lane;
            v[u] = t < T ? __ldg(in + off + (rho + t * g) * es) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int64_t t = t0 + u * 32 + lane;
            uint64_t sc = sat_add(warp_incl_scan_sat(v[u], lane), carry);
            const int64_t x = off + (rho + t * g) * es;
            if (t < T) out[x] = x < ones_below ? 1ull : sc;
            carry = shfl_u64(sc, 31);
        }
    }
}

constexpr int SCAN_MINB_DEFAULT = 4;

// MINB: CTAs per SM the register budget is set for (3 fit without a bound:
// 76 registers; 4 at 64 registers; 6 at 40 registers with a few spills).
template <int MINB>
__global__ void __launch_bounds__(THREADS, MINB) scan_tasks_kernel(const ScanJob *__restrict__ jobs,
                                                                   const ScanTask *__restrict__ tasks) {
    const ScanTask t = tasks[blockIdx.x];
    const ScanJob J = jobs[t.job];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int64_t es = J.es ? J.es : 1, off = J.off;
    switch (t.kind) {
        case TK_DIRECT:
            for (int64_t rho = t.begin + warp; rho < t.end; rho += nwarps)
                chain_scan_warp(J.in, J.out, J.len, J.g, rho, lane, J.ones_below, off, es);
            break;
        case TK_LANES: {
            // lane l of warp w: chain rho = begin + 32 w + l, walked down with
            // its own running sum; a warp's loads and stores cover 32
            // neighbouring entries of a row (one 256-byte span when es = 1)
            const int64_t rho = t.begin + (int64_t)warp * 32 + lane;
            if (rho >= t.end) break;
            const uint64_t *__restrict__ in = J.in;
            uint64_t *__restrict__ out = J.out;
            const int64_t T = (J.len - rho + J.g - 1) / J.g;
            uint64_t acc = 0;
            for (int64_t t0 = 0; t0 < T; t0 += LANE_ILP) {
                uint64_t v[LANE_ILP];
#pragma unroll
                for (int u = 0; u < LANE_ILP; ++u)
                    v[u] = t0 + u < T ? __ldg(in + off + (rho + (t0 + u) * J.g) * es) : 0ull;
#pragma unroll
                for (int u = 0; u < LANE_ILP; ++u) {
                    if (t0 + u < T) {
                        const int64_t x = off + (rho + (t0 + u) * J.g) * es;
                        acc = sat_add(acc, v[u]);
                        out[x] = x < J.ones_below ? 1ull : acc;
                    }
                }
            }
            break;
        }
        case TK_SSCAN:
            for (int64_t rho = t.begin + warp; rho < t.end; rho += nwarps)
                chain_scan_warp(J.S, J.Sincl, J.slen, J.g, rho, lane);
            break;
        case TK_BSUM: {
            const int64_t rb = J.rb > 0 ? J.rb : RB;
            for (int64_t i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
                const int64_t b = i / J.g, rho = i - b * J.g;
                const int64_t r0 = (b * rb) * J.g + rho;
                uint64_t acc = 0;
                for (int64_t u0 = 0; u0 < rb; u0 += 8) {
                    uint64_t v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int64_t r = r0 + (u0 + u) * J.g;
                        v[u] = (u0 + u < rb && r < J.len) ? __ldg(J.in + off + r * es) : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc = sat_add(acc, v[u]);
                }
                J.S[i] = acc;
            }
            break;
        }
        case TK_APPLY: {
            const int64_t rb = J.rb > 0 ? J.rb : RB;
            for (int64_t i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
                const int64_t b = i / J.g, rho = i - b * J.g;
                uint64_t acc = b > 0 ? J.Sincl[i - J.g] : 0ull;
                const int64_t r0 = (b * rb) * J.g + rho;
                for (int64_t u0 = 0; u0 < rb; u0 += 8) {
                    uint64_t v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int64_t r = r0 + (u0 + u) * J.g;
                        v[u] = (u0 + u < rb && r < J.len) ? __ldg(J.in + off + r * es) : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int64_t r = r0 + (u0 + u) * J.g;
                        if (u0 + u < rb && r < J.len) {
                            const int64_t x = off + r * es;
                            acc = sat_add(acc, v[u]);
                            J.out[x] = x < J.ones_below ? 1ull : acc;
                        }
                    }
                }
            }
            break;
        }
        case TK_DELTA:
            for (int64_t i = t.begin + threadIdx.x; i < t.end; i += blockDim.x)
                J.out[off + i * es] = (off + i * es == 0) ? 1ull : 0ull;
            break;
        case TK_ONES:
            for (int64_t i = t.begin + threadIdx.x; i < t.end; i += blockDim.x)
                J.out[off + i * es] = 1ull;
            break;
        case TK_PAIR:
            // |Z(r, (g, h))|: the a with g a = r (mod h) in [0, r / g] are
            // a = a* (mod h1), a* = (r / e) inv (mod h1), when e divides r
            // (row d-1 is written only for whole rows: es == 1)
            // (32-bit: entries, generators and their quotients are below
            // 2^31; the product (re mod h1) inv needs 64 bits when h1 >= 2^16)
            {
                const uint32_t e = (uint32_t)J.e, h1 = (uint32_t)J.h1, g1 = (uint32_t)J.g1;
                const uint32_t h = (uint32_t)J.h, inv = (uint32_t)J.inv;
                const bool small = h1 < 65536u;
                for (int64_t i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
                    const uint32_t r = (uint32_t)(off + i * es);
                    uint64_t c = 0;
                    if (r % e == 0) {
                        const uint32_t re = r / e;
                        const uint32_t astar =
                            small ? (re % h1) * inv % h1
                                  : (uint32_t)((uint64_t)(re % h1) * inv % h1);
                        const uint32_t q = re / g1;
                        c = q >= astar ? (uint64_t)((q - astar) / h1 + 1) : 0ull;
                    }
                    J.out[r] = c;
                    if (J.ones_below && es == 1) J.out[J.len + r] = (r % h == 0) ? 1ull : 0ull;
                }
            }
            break;
        case TK_LINEAR:
            for (int64_t i = t.begin + threadIdx.x; i < t.end; i += blockDim.x) {
                const int64_t x = off + i * es;
                J.out[x] = x < J.ones_below ? 1ull : (uint64_t)((uint32_t)x / (uint32_t)J.g + 1u);
            }
            break;
        default:
            break;
    }
}

// FZ_SCAN_MINB=1|4|6: the register budget of the batched scans (tuning only).
static int scan_minb() {
    static const int v = [] {
        const char *e = getenv("FZ_SCAN_MINB");
        const int x = e ? atoi(e) : 0;
        return (x == 1 || x == 4 || x == 6) ? x : SCAN_MINB_DEFAULT;
    }();
    return v;
}

int launch_scan_tasks(const ScanJob *jobs, const ScanTask *tasks, int ntasks, cudaStream_t s) {
    if (ntasks <= 0) return FZ_OK;
    switch (scan_minb()) {
        case 1: scan_tasks_kernel<1><<<ntasks, THREADS, 0, s>>>(jobs, tasks); break;
        case 6: scan_tasks_kernel<6><<<ntasks, THREADS, 0, s>>>(jobs, tasks); break;
        default: scan_tasks_kernel<4><<<ntasks, THREADS, 0, s>>>(jobs, tasks); break;
    }
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

int64_t scan_direct_limit() { return DIRECT_T; }
// Block sums a task of a blocked scan covers: one a thread (256).
// FZ_SCAN_BS_TASK=2048 gives a thread eight (tuning only).
int64_t scan_blocks_per_task() {
    static const int64_t v = [] {
        const char *e = getenv("FZ_SCAN_BS_TASK");
        const long x = e ? atol(e) : 0;
        return (x >= 256 && x <= 65536 && x % 256 == 0) ? (int64_t)x : (int64_t)THREADS;
    }();
    return v;
}

// FZ_SCAN_LANES=0 scans every short chain with a warp (tuning only).
int64_t scan_lane_limit() {
    static const int64_t v = [] {
        const char *e = getenv("FZ_SCAN_LANES");
        return (e && strcmp(e, "0") == 0) ? (int64_t)0 : LANE_T;
    }();
    return v;
}
int scan_block_rows() { return RB; }

int launch_count_rolling(const int32_t *g, int d, int32_t n, uint64_t *a, uint64_t *b,
                         uint64_t *tmp, uint64_t **result, cudaStream_t s) {
    const int64_t len = (int64_t)n + 1;
    row_delta_kernel<<<grid_for(len, THREADS), THREADS, 0, s>>>(a, len);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    uint64_t *below = a, *cur = b;
    for (int j = d - 1; j >= 0; --j) {
        int rc = strided_scan(below, cur, len, g[j], tmp, s);
        if (rc != FZ_OK) return rc;
        uint64_t *t = below;
        below = cur;
        cur = t;
    }
    *result = below;
    return FZ_OK;
}

// in: len entries; out: len + 1 entries, out[0] = 0, out[r+1] = sum_{r' <= r} in[r'].
int launch_exclusive_scan_tmp(const uint64_t *in, uint64_t *out, int64_t len, uint64_t *tmp,
                              cudaStream_t s) {
    FZ_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    return strided_scan(in, out + 1, len, 1, tmp, s);
}

// ---------------------------------------------------------------------------
// Write probe (fz_write_probe): distinct words, 16-byte stores, a grid of
// 8 CTAs of 256 threads per SM striding over the buffer.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) write_probe_kernel(int4 *__restrict__ out, uint64_t n16,
                                                          int32_t *__restrict__ tail,
                                                          uint64_t tail_words, uint64_t tail_w0) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const int32_t w = (int32_t)(i * 4);
        out[i] = make_int4(w, w + 1, w + 2, w + 3);
    }
    if (blockIdx.x == 0 && threadIdx.x < tail_words)
        tail[threadIdx.x] = (int32_t)(tail_w0 + threadIdx.x);
}

int launch_write_probe(int32_t *out, uint64_t words, cudaStream_t s) {
    int dev = 0, sms = 1;
    FZ_CUDA_TRY(cudaGetDevice(&dev));
    FZ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint64_t n16 = words / 4;
    const uint64_t tail_words = words - n16 * 4;  // < 4
    uint64_t grid = (uint64_t)sms * 8;
    const uint64_t want = (n16 + 255) / 256;
    if (want < grid) grid = want < 1 ? 1 : want;
    write_probe_kernel<<<(unsigned)grid, 256, 0, s>>>(reinterpret_cast<int4 *>(out), n16,
                                                      out + n16 * 4, tail_words, n16 * 4);
    note_launch();
    FZ_CUDA_TRY(cudaGetLastError());
    return FZ_OK;
}

}  // namespace fz
