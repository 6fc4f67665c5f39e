// fz_memo.cu -- the memo of tail sets, built by the dynamic
// FactorizationsUpToElement pass of Section 2.
//
// For a tail (t_0..t_{k-1}) and top, Memo[r] = Z(r, tail) for r = 0..top-1,
// each list in descending lexicographic order, stored as a CSR (offsets O,
// k int32 per row).  The lists come from the disjoint, lexicographically
// ordered recurrence (Lemma "disjlex", Section 2.1):
//
//   Z(m) = incr_0(Z_{>=0}(m - t_0)) ++ ... ++ incr_{k-1}(Z_{>=k-1}(m - t_{k-1}))
//
// where Z_{>=i}(x), the rows of Z(x) with zeros left of i, is the last
// |Z_{>=i}(x)| = Ct[i][x] rows of Z(x).  Saving those cardinalities (Section
// 2.3) pre-assigns every copy its source and destination; this build writes
// the assignment out as a gather map (one entry per memo row: source row and
// incremented coordinate) in a fully parallel pre-pass.  The copies then run
// elementwise in batches of b = min(tail) consecutive elements (Section 2.2):
// elements m+1..m+b depend only on elements <= m, so every batch is one
// parallel copy-and-increment step (the kernel copyAndIncrementIndex of
// Section 2.4), and batches are separated by a bounded grid barrier inside one
// cooperative launch.  Empty batches need no barrier.
#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr uint64_t MAP_ZERO = ~0ull;  // the row of Z(0): all zeros
constexpr int THREADS = 256;

struct MapParams {
    const uint64_t *Ct;  // tail count table rows 0..k, stride cs
    int64_t cs;
    const uint64_t *O;
    uint64_t *map;
    int *status;
    int top;
    int k;
    int t[FZ_MAX_D];
};

// One warp per element m: lay out the blocks incr_i(Z_{>=i}(m - t_i)).
__global__ void __launch_bounds__(THREADS) memo_map_kernel(MapParams P) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t m = warp; m < P.top; m += nwarps) {
        uint64_t dst = __ldg(P.O + m);
        const uint64_t end = __ldg(P.O + m + 1);
        if (m == 0) {
            if (lane == 0 && end == dst + 1) P.map[dst] = MAP_ZERO;
            if (lane == 0 && end != dst + 1) atomicExch(P.status, (int)DEV_INTERNAL);
            continue;
        }
        for (int i = 0; i < P.k; ++i) {
            const int64_t src_m = m - (int64_t)P.t[i];
            if (src_m < 0) continue;
            const uint64_t len = __ldg(P.Ct + (int64_t)i * P.cs + src_m);
            if (len == 0) continue;
            const uint64_t src = __ldg(P.O + src_m + 1) - len;  // suffix Z_{>=i}(src_m)
            if (dst + len > end) {  // bounds guard: the counts must tile Z(m) exactly
                if (lane == 0) atomicExch(P.status, (int)DEV_INTERNAL);
                break;
            }
            for (uint64_t r = lane; r < len; r += 32)
                P.map[dst + r] = ((src + r) << 4) | (uint64_t)i;
            dst += len;
        }
        if (lane == 0 && dst != end) atomicExch(P.status, (int)DEV_INTERNAL);
    }
}

struct FillParams {
    const uint64_t *O;
    const uint64_t *map;
    int32_t *rows;
    int *status;
    GridBarrier bar;
    int top;
    int k;
    int b;        // elements per batch
    int nbatch;
};

// Batches of b elements; one copy-and-increment per memo row; bounded grid
// barrier between non-empty batches.
__global__ void __launch_bounds__(THREADS) memo_fill_kernel(FillParams P) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int k = P.k;
    for (int q = 0; q < P.nbatch; ++q) {
        const int64_t m0 = (int64_t)q * P.b;
        int64_t m1 = m0 + P.b;
        if (m1 > P.top) m1 = P.top;
        const uint64_t R0 = __ldg(P.O + m0), R1 = __ldg(P.O + m1);
        if (R1 == R0) continue;
        for (uint64_t R = R0 + tid; R < R1; R += nthreads) {
            const uint64_t e = __ldg(P.map + R);
            int32_t *dst = P.rows + R * k;
            if (e == MAP_ZERO) {
                for (int c = 0; c < k; ++c) dst[c] = 0;
            } else if ((e >> 4) >= R0) {  // bounds guard: sources precede the batch
                atomicExch(P.status, (int)DEV_INTERNAL);
            } else {
                const int inc = (int)(e & 15u);
                const int32_t *src = P.rows + (e >> 4) * k;
                for (int c = 0; c < k; ++c) {
                    int32_t v = ld_cg_s32(src + c);
                    dst[c] = v + (c == inc ? 1 : 0);
                }
            }
        }
        if (q + 1 < P.nbatch && !grid_barrier(P.bar, P.status)) return;
    }
}

int coop_grid(const void *kernel, int threads) {
    DeviceProps dp;
    if (device_props(&dp) != FZ_OK) return -1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) !=
        cudaSuccess)
        return -1;
    if (per_sm < 1) return -1;
    if (per_sm > 2) per_sm = 2;
    return per_sm * dp.sms;
}

}  // namespace

int launch_memo_build(const int32_t *tail, int k, int32_t top, uint64_t rows,
                      const MemoBuffers &mb, cudaStream_t s) {
    if (top <= 0 || rows == 0) return FZ_OK;
    if (!mb.Ct || !mb.O || !mb.map || !mb.rows || !mb.status || !mb.bar)
        return set_error(FZ_EINTERNAL, "memo build: missing device buffer");
    MapParams mp{};
    mp.Ct = mb.Ct;
    mp.cs = mb.cs;
    mp.O = mb.O;
    mp.map = mb.map;
    mp.status = mb.status;
    mp.top = top;
    mp.k = k;
    int tmin = tail[0];
    for (int i = 0; i < k; ++i) {
        mp.t[i] = tail[i];
        if (tail[i] < tmin) tmin = tail[i];
    }
    {
        int64_t warps = top;
        int64_t blocks = (warps * 32 + THREADS - 1) / THREADS;
        if (blocks > 4096) blocks = 4096;
        memo_map_kernel<<<(int)blocks, THREADS, 0, s>>>(mp);
        note_launch();
        FZ_CUDA_TRY(cudaGetLastError());
    }
    FillParams fp{};
    fp.O = mb.O;
    fp.map = mb.map;
    fp.rows = mb.rows;
    fp.status = mb.status;
    fp.bar.count = mb.bar;
    fp.bar.gen = mb.bar + 1;
    fp.top = top;
    fp.k = k;
    fp.b = tmin;
    fp.nbatch = (int)(((int64_t)top + tmin - 1) / tmin);
    int grid = coop_grid((const void *)memo_fill_kernel, THREADS);
    if (grid <= 0) return set_error(FZ_ECUDA, "memo build: no cooperative occupancy");
    FZ_CUDA_TRY(cudaMemsetAsync(mb.bar, 0, sizeof(unsigned), s));
    void *args[] = {&fp};
    FZ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)memo_fill_kernel, dim3(grid),
                                            dim3(THREADS), args, 0, s));
                                            note_launch();
    return FZ_OK;
}

}  // namespace fz
