// k_batch.cu -- many compressed-matrix operations of mixed kinds and sizes as
// one persistent, graph-captured launch.
//
// The block-wise algorithms of Sec. III of "Compressed Matrix Computations"
// (arXiv 2202.13007) make every operation a set of independent per-block
// tasks.  The plan cuts each operation into work items (a range of 8x8
// blocks, or one 64x64 DMMA tile of a matrix product); persistent CTAs take
// items from a device queue in order.  The per-block code is the same device
// code as the single-operation kernels (block_codec.cuh, block_ops.cuh,
// gemm_fp64.cuh).
//
// Queue order makes the one dependency safe: the decompression items of all
// matrix products come first, their 64x64 product tiles last; a CTA that takes
// a tile waits (bounded) until the counter of its product's decompression
// items is complete, and those items were all taken earlier by running CTAs.
#include <algorithm>
#include <cstring>
#include <vector>

#include "batch_internal.cuh"
#include "block_codec.cuh"
#include "block_ops.cuh"
#include "compress_fix.cuh"
#include "gemm_fp64.cuh"

namespace blaz {

__device__ int g_batch_status;  // BLAZ_ERR_TIMEOUT when a tile's wait ran out

namespace batch {

constexpr int kThreads = kGemmThreads;  // 128: also the thread count of a DMMA tile
constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ double cta_sum128(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < kThreads / 32; ++q) r += red[q];
    __syncthreads();
    return r;
}

// The exact fix-up of one block by a team of 8 lanes (compress_fix.cuh),
// kept out of line: it is rare, and inlined it would raise the register
// pressure of every path of the batch kernel.
__device__ __noinline__ void batch_fix(const double *A, int64_t lda, int64_t rows, int64_t cols, int64_t nbc,
                                       int64_t b, uint32_t pending, double *s, uint8_t *phi, int8_t *code, int u,
                                       int tbase, unsigned tmask)
{
    if (pending == kPendingAll)
        fix_whole_block<false>(A, lda, rows, cols, nbc, b, s, phi, code, u, tbase, tmask);
    else
        fix_codes_of_block<false>(A, lda, rows, cols, nbc, b, pending, s, phi, code, u, tbase, tmask);
}

__global__ void __launch_bounds__(kThreads)
    k_batch(const DevOp *__restrict__ ops, const Item *__restrict__ items, int nitems, unsigned *next,
            unsigned *done, double *partials)
{
    __shared__ GemmSmem gs;
    __shared__ double red[kThreads / 32];
    __shared__ int s_item, s_ok;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const Item w = items[it];
        const DevOp &op = ops[w.op];
        if (w.tile) {
            // 64 x 64 tile of a product: wait for the op's decompression items.
            if (tid == 0) {
                const bool ok = bounded_wait_geq(&done[w.op], (unsigned)op.nitems, kWaitCycles);
                if (!ok) atomicExch(&g_batch_status, BLAZ_ERR_TIMEOUT);
                __threadfence();
                s_ok = ok;
            }
            __syncthreads();
            if (s_ok)
                gemm_tile_fp64<true>(gs, op.scratch, op.k, op.B, op.ldb, op.C, op.ldc, op.n, op.k, op.m, w.b0, w.b1);
            __syncthreads();
            continue;
        }
        switch (op.kind) {
        case BLAZ_OP_COMPRESS: {
            // One block per lane with a warp-uniform trip count, then the
            // blocks the certified pass left undecided are evaluated exactly by
            // teams of 8 lanes (four blocks per round), as in k_compress_fix.
            const int lane = tid & 31, u = lane & 7, tbase = lane & ~7, team = lane >> 3;
            const unsigned tmask = 0xFFu << tbase;
            const int64_t cols = op.nbc * 8, rows = INT64_MAX / 16;  // no partial blocks in a batch
            for (int64_t bb = w.b0 + (tid & ~31); bb < w.b1; bb += kThreads) {
                const int64_t b = bb + lane;
                uint32_t pending = 0;
                if (b < w.b1) {
                    const int64_t bi = b / op.nbc, bj = b - bi * op.nbc;
                    double d[64];
                    if (op.vec) load_block<true>(op.A, op.lda, bi, bj, d);
                    else load_block<false>(op.A, op.lda, bi, bj, d);
                    op.fo[b] = d[0];
                    double sv;
                    uint8_t ph;
                    int8_t c[kKeep];
                    pending = compress_block_fast(d, sv, ph, c);
                    op.so[b] = sv;
                    if (pending != kPendingAll) {
                        op.po[b] = ph;
                        store_codes(op.co + b * kKeep, c);
                    }
                }
                unsigned need = __ballot_sync(0xffffffffu, pending != 0u);
                if (!need) continue;
                __syncwarp();  // s, phi and the decided codes are visible to the whole warp
                while (need) {
                    unsigned m = need;
                    for (int k = 0; k < team; ++k) m &= m - 1;
                    const int target = m ? __ffs(m) - 1 : -1;
                    const uint32_t pend = __shfl_sync(0xffffffffu, pending, target < 0 ? 0 : target);
                    if (target >= 0)
                        batch_fix(op.A, op.lda, rows, cols, op.nbc, bb + target, pend, op.so, op.po, op.co, u, tbase,
                                  tmask);
                    for (int k = 0; k < 4; ++k) need &= need - 1;
                    __syncwarp();
                }
            }
            break;
        }
        case BLAZ_OP_DECOMPRESS:
        case BLAZ_OP_MATMUL: {
            double *dst = op.kind == BLAZ_OP_MATMUL ? op.scratch : op.C;
            const int64_t ld = op.kind == BLAZ_OP_MATMUL ? op.k : op.ldc;
            for (int64_t b = w.b0 + tid; b < w.b1; b += kThreads) {
                const int64_t bi = b / op.nbc, bj = b - bi * op.nbc;
                double out[64];
                decompress_block_at(op.fa[b], op.sa[b], op.pa[b], op.ca + b * kKeep, out);
                double *p = dst + (bi * 8) * ld + bj * 8;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) p[i * ld + j] = out[i * 8 + j];
            }
            if (op.kind == BLAZ_OP_MATMUL) {
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    atomicAdd(&done[w.op], 1u);
                }
            }
            break;
        }
        case BLAZ_OP_ADD:
            for (int64_t b = w.b0 + tid; b < w.b1; b += kThreads)
                add_block_fast<false>(b, op.fa, op.sa, op.pa, op.ca, op.fb, op.sb, op.pb, op.cb, op.fo, op.so, op.po, op.co);
            break;
        case BLAZ_OP_SUB:
            for (int64_t b = w.b0 + tid; b < w.b1; b += kThreads)
                add_block_fast<true>(b, op.fa, op.sa, op.pa, op.ca, op.fb, op.sb, op.pb, op.cb, op.fo, op.so, op.po, op.co);
            break;
        case BLAZ_OP_SCALE: {
            const bool copy = (op.po != op.pa) || (op.co != op.ca);
            for (int64_t b = w.b0 + tid; b < w.b1; b += kThreads)
                scale_block(b, op.fa, op.sa, op.pa, op.ca, op.c, op.fo, op.so, op.po, op.co, copy);
            break;
        }
        case BLAZ_OP_DOT: {
            double acc = 0.0;
            for (int64_t b = w.b0 + tid; b < w.b1; b += kThreads) {
                double x[64], y[64];
                decompress_block_at(op.fa[b], op.sa[b], op.pa[b], op.ca + b * kKeep, x);
                decompress_block_at(op.fb[b], op.sb[b], op.pb[b], op.cb + b * kKeep, y);
                double blk = 0.0;
#pragma unroll
                for (int p = 0; p < 64; ++p) blk = fma(x[p], y[p], blk);
                acc += blk;
            }
            const double tot = cta_sum128(acc, red);
            if (tid == 0) {
                partials[op.partial_base + (it - op.first_item)] = tot;
                __threadfence();
                s_ok = (atomicAdd(&done[w.op], 1u) == (unsigned)op.nitems - 1);
            }
            __syncthreads();
            if (s_ok) {  // last item of this dot: sum the partials in item order
                __threadfence();
                double v = 0.0;
                for (int q = tid; q < op.nitems; q += kThreads) v += __ldcg(partials + op.partial_base + q);
                const double r = cta_sum128(v, red);
                if (tid == 0) *op.result = r;
            }
            break;
        }
        default:
            break;
        }
        __syncthreads();
    }
}

int launch(const DevOp *d_ops, const Item *d_items, int nitems, unsigned *d_counters, double *d_partials, int grid,
           cudaStream_t st)
{
    if (nitems <= 0) return BLAZ_OK;
    k_batch<<<grid, kThreads, 0, st>>>(d_ops, d_items, nitems, d_counters, d_counters + 1, d_partials);
    return launch_status();
}

}  // namespace batch

int batch_device_status()
{
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_batch_status, sizeof(int));
    if (e != cudaSuccess) return set_cuda_error(e);
    if (v != 0) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_batch_status, &zero, sizeof(int));
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return v;
}

}  // namespace blaz

using namespace blaz;

struct blaz_plan {
    int device = 0;
    std::vector<blaz_op> ops;
    blaz_batch_cfg cfg{};
    batch::DevOp *d_ops = nullptr;
    batch::Item *d_items = nullptr;
    unsigned *d_counters = nullptr;  // [0]: next item, [1 + op]: per-op done counter
    double *d_partials = nullptr;
    char *d_scratch = nullptr;       // decompressed operands of the products
    size_t scratch_bytes = 0, cap_items = 0, cap_partials = 0;
    int nitems = 0, ngemm = 0, grid = 0;
    double tuned_ms = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {
int64_t nblk(const blaz_cmat &m) { return (m.rows / 8) * (m.cols / 8); }
}  // namespace

int blaz::batch::check_op(const blaz_op &o)
{
    int rc;
    switch (o.kind) {
    case BLAZ_OP_COMPRESS:
        if ((rc = validate_cmat(&o.out))) return rc;
        if (nblk(o.out) && !o.A) return BLAZ_ERR_NULL;
        if (nblk(o.out) && o.lda < o.out.cols) return BLAZ_ERR_LD;
        return BLAZ_OK;
    case BLAZ_OP_DECOMPRESS:
        if ((rc = validate_cmat(&o.a))) return rc;
        if (nblk(o.a) && !o.C) return BLAZ_ERR_NULL;
        if (nblk(o.a) && o.ldc < o.a.cols) return BLAZ_ERR_LD;
        return BLAZ_OK;
    case BLAZ_OP_ADD:
    case BLAZ_OP_SUB:
        if ((rc = validate_cmat(&o.a)) || (rc = validate_cmat(&o.b)) || (rc = validate_cmat(&o.out))) return rc;
        if (o.a.rows != o.b.rows || o.a.cols != o.b.cols || o.a.rows != o.out.rows || o.a.cols != o.out.cols)
            return BLAZ_ERR_SHAPE;
        return BLAZ_OK;
    case BLAZ_OP_SCALE:
        if ((rc = validate_cmat(&o.a)) || (rc = validate_cmat(&o.out))) return rc;
        if (o.a.rows != o.out.rows || o.a.cols != o.out.cols) return BLAZ_ERR_SHAPE;
        return BLAZ_OK;
    case BLAZ_OP_DOT:
        if ((rc = validate_cmat(&o.a)) || (rc = validate_cmat(&o.b))) return rc;
        if (o.a.rows != o.b.rows || o.a.cols != o.b.cols) return BLAZ_ERR_SHAPE;
        if (!o.result) return BLAZ_ERR_NULL;
        return BLAZ_OK;
    case BLAZ_OP_MATMUL:
        if ((rc = validate_cmat(&o.a))) return rc;
        if (o.m < 0) return BLAZ_ERR_SHAPE;
        if (o.a.rows && o.m && (!o.C || (o.a.cols && !o.B))) return BLAZ_ERR_NULL;
        if (o.a.rows && o.m && (o.ldc < o.m || (o.a.cols && o.ldb < o.m))) return BLAZ_ERR_LD;
        return BLAZ_OK;
    default:
        return BLAZ_ERR_ARG;
    }
}

namespace {

// Output and input base pointers of an op (for the autotune aliasing check).
void op_ptrs(const blaz_op &o, std::vector<const void *> &in, std::vector<const void *> &out)
{
    auto cm = [](const blaz_cmat &m, std::vector<const void *> &v) {
        if (m.f) v.push_back(m.f);
        if (m.s) v.push_back(m.s);
        if (m.phi) v.push_back(m.phi);
        if (m.code) v.push_back(m.code);
    };
    switch (o.kind) {
    case BLAZ_OP_COMPRESS: in.push_back(o.A); cm(o.out, out); break;
    case BLAZ_OP_DECOMPRESS: cm(o.a, in); out.push_back(o.C); break;
    case BLAZ_OP_ADD:
    case BLAZ_OP_SUB: cm(o.a, in); cm(o.b, in); cm(o.out, out); break;
    case BLAZ_OP_SCALE: cm(o.a, in); cm(o.out, out); break;
    case BLAZ_OP_DOT: cm(o.a, in); cm(o.b, in); out.push_back(o.result); break;
    case BLAZ_OP_MATMUL: cm(o.a, in); in.push_back(o.B); out.push_back(o.C); break;
    }
}

}  // namespace

void blaz::batch::build_work(const blaz_op *ops, int nops, int64_t bpi, char *scratch, std::vector<DevOp> &dops,
                             std::vector<Item> &all, int64_t &partials, size_t &scratch_bytes_out, int &ngemm)
{
    dops.assign(nops, DevOp{});
    std::vector<Item> first, middle, tiles;
    partials = 0;
    size_t sbytes = 0;
    std::vector<size_t> scratch_off(nops, 0);
    for (int i = 0; i < nops; ++i) {
        const blaz_op &o = ops[i];
        if (o.kind == BLAZ_OP_MATMUL && o.a.rows && o.m) {
            scratch_off[i] = sbytes;
            sbytes += ((size_t)(o.a.rows * o.a.cols) * 8 + 255) & ~(size_t)255;
        }
    }
    scratch_bytes_out = sbytes;
    for (int i = 0; i < nops; ++i) {
        const blaz_op &o = ops[i];
        DevOp &d = dops[i];
        std::memset(&d, 0, sizeof(d));
        d.kind = o.kind;
        const blaz_cmat &drive = (o.kind == BLAZ_OP_COMPRESS) ? o.out : o.a;
        d.nbc = drive.cols / 8;
        const int64_t nb = nblk(drive);
        d.fa = o.a.f; d.sa = o.a.s; d.pa = o.a.phi; d.ca = o.a.code;
        d.fb = o.b.f; d.sb = o.b.s; d.pb = o.b.phi; d.cb = o.b.code;
        d.fo = o.out.f; d.so = o.out.s; d.po = o.out.phi; d.co = o.out.code;
        d.A = o.A; d.lda = o.lda;
        d.vec = ((uintptr_t)o.A % 16 == 0) && (o.lda % 2 == 0);
        d.c = o.c;
        d.result = o.result;
        d.B = o.B; d.ldb = o.ldb; d.m = o.m;
        d.C = o.C; d.ldc = o.ldc;
        d.n = o.a.rows; d.k = o.a.cols;
        if (o.kind == BLAZ_OP_MATMUL) {
            if (!o.a.rows || !o.m) continue;                   // empty product: nothing to do
            d.scratch = scratch ? (double *)(scratch + scratch_off[i]) : nullptr;
        }
        std::vector<Item> &dst = (o.kind == BLAZ_OP_MATMUL) ? first : middle;
        d.first_item = (int32_t)dst.size();
        int cnt = 0;
        for (int64_t b0 = 0; b0 < nb; b0 += bpi) {
            dst.push_back({i, 0, b0, std::min(nb, b0 + bpi)});
            ++cnt;
        }
        if (o.kind == BLAZ_OP_DOT && cnt == 0) {  // empty dot: one item that writes 0
            dst.push_back({i, 0, 0, 0});
            cnt = 1;
        }
        d.nitems = cnt;
        if (o.kind == BLAZ_OP_DOT) {
            d.partial_base = partials;
            partials += cnt;
        }
        if (o.kind == BLAZ_OP_MATMUL)
            for (int64_t r = 0; r < o.a.rows; r += kGemmBM)
                for (int64_t c = 0; c < o.m; c += kGemmBN) tiles.push_back({i, 1, r, c});
    }
    const int off = (int)first.size();
    for (int i = 0; i < nops; ++i)
        if (ops[i].kind != BLAZ_OP_MATMUL) dops[i].first_item += off;
    all.clear();
    all.reserve(first.size() + middle.size() + tiles.size());
    all.insert(all.end(), first.begin(), first.end());
    all.insert(all.end(), middle.begin(), middle.end());
    all.insert(all.end(), tiles.begin(), tiles.end());
    ngemm = (int)tiles.size();
}

namespace {

// Build the device descriptors and the work list of a plan for a configuration.
int build(blaz_plan *p, const blaz_batch_cfg &cfg)
{
    const int64_t bpi = cfg.blocks_per_item > 0 ? cfg.blocks_per_item : 256;
    const int nops = (int)p->ops.size();
    std::vector<batch::DevOp> dops;
    std::vector<batch::Item> all;
    int64_t partials = 0;
    size_t scratch = 0;
    int ngemm = 0;
    batch::build_work(p->ops.data(), nops, bpi, nullptr, dops, all, partials, scratch, ngemm);
    if (scratch > p->scratch_bytes) {
        if (p->d_scratch) cudaFree(p->d_scratch);
        p->d_scratch = nullptr;
        cudaError_t e = cudaMalloc(&p->d_scratch, scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p->scratch_bytes = 0;
            return e == cudaErrorMemoryAllocation ? BLAZ_ERR_OOM : set_cuda_error(e);
        }
        p->scratch_bytes = scratch;
    }
    batch::build_work(p->ops.data(), nops, bpi, p->d_scratch, dops, all, partials, scratch, ngemm);
    if (all.size() > 0x7fffffff) return BLAZ_ERR_ARG;
    cudaError_t e;
    if (!p->d_ops) {
        if ((e = cudaMalloc(&p->d_ops, sizeof(batch::DevOp) * std::max(1, nops))) != cudaSuccess) return set_cuda_error(e);
        if ((e = cudaMalloc(&p->d_counters, sizeof(unsigned) * (1 + std::max(1, nops)))) != cudaSuccess)
            return set_cuda_error(e);
    }
    if (all.size() > p->cap_items) {
        if (p->d_items) cudaFree(p->d_items);
        if ((e = cudaMalloc(&p->d_items, sizeof(batch::Item) * std::max<size_t>(1, all.size()))) != cudaSuccess)
            return set_cuda_error(e);
        p->cap_items = all.size();
    }
    if ((size_t)partials > p->cap_partials) {
        if (p->d_partials) cudaFree(p->d_partials);
        if ((e = cudaMalloc(&p->d_partials, sizeof(double) * std::max<int64_t>(1, partials))) != cudaSuccess)
            return set_cuda_error(e);
        p->cap_partials = partials;
    }
    if (nops && (e = cudaMemcpy(p->d_ops, dops.data(), sizeof(batch::DevOp) * nops, cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
        return set_cuda_error(e);
    if (!all.empty() &&
        (e = cudaMemcpy(p->d_items, all.data(), sizeof(batch::Item) * all.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
        return set_cuda_error(e);
    p->nitems = (int)all.size();
    p->ngemm = ngemm;
    const int cps = cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : 2;
    p->grid = std::max(1, std::min<int>(num_sms() * cps, std::max(1, p->nitems)));
    p->cfg = cfg;
    p->cfg.blocks_per_item = (int32_t)bpi;
    p->cfg.ctas_per_sm = cps;

    // Capture: reset the counters, then the persistent launch.
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return set_cuda_error(e);
    int rc = BLAZ_OK;
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) rc = set_cuda_error(e);
    if (!rc) {
        cudaMemsetAsync(p->d_counters, 0, sizeof(unsigned) * (1 + std::max(1, nops)), cap);
        batch::launch(p->d_ops, p->d_items, p->nitems, p->d_counters, p->d_partials, p->grid, cap);
        e = cudaStreamEndCapture(cap, &p->graph);
        if (e != cudaSuccess) rc = set_cuda_error(e);
    }
    if (!rc && (e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess) rc = set_cuda_error(e);
    cudaStreamDestroy(cap);
    return rc;
}

}  // namespace

extern "C" {

int blaz_batch_plan(const blaz_op *ops, int64_t nops, const blaz_batch_cfg *cfg, blaz_plan **plan, void *stream)
{
    if (!plan || (nops > 0 && !ops)) return BLAZ_ERR_NULL;
    if (nops < 0) return BLAZ_ERR_ARG;
    *plan = nullptr;
    for (int64_t i = 0; i < nops; ++i) {
        int rc = batch::check_op(ops[i]);
        if (rc) return rc;
    }
    blaz_batch_cfg c = cfg ? *cfg : blaz_batch_cfg{0, 0, 0};
    if (c.blocks_per_item < 0 || c.ctas_per_sm < 0 || c.ctas_per_sm > 32) return BLAZ_ERR_ARG;
    if (c.autotune) {
        std::vector<const void *> in, out;
        for (int64_t i = 0; i < nops; ++i) op_ptrs(ops[i], in, out);
        std::sort(in.begin(), in.end());
        for (const void *o : out)
            if (std::binary_search(in.begin(), in.end(), o)) return BLAZ_ERR_ARG;
    }
    blaz_plan *p = new blaz_plan();
    cudaGetDevice(&p->device);
    p->ops.assign(ops, ops + nops);
    int rc = BLAZ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (c.autotune && nops > 0) {
        const int bpis[] = {64, 128, 256, 512, 1024};
        const int cpss[] = {1, 2};
        double best = 1e30;
        blaz_batch_cfg best_cfg{256, 2, 0};
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int bpi : bpis)
            for (int cps : cpss) {
                blaz_batch_cfg t{bpi, cps, 0};
                if ((rc = build(p, t))) break;
                cudaGraphLaunch(p->exec, st);  // warm-up
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3; ++r) cudaGraphLaunch(p->exec, st);
                cudaEventRecord(e1, st);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    rc = set_cuda_error(e);
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms / 3 < best) {
                    best = ms / 3;
                    best_cfg = t;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!rc) {
            rc = build(p, best_cfg);
            p->tuned_ms = best;
            p->cfg.autotune = 1;
        }
    } else {
        rc = build(p, c);
    }
    if (rc) {
        blaz_batch_free(p);
        return rc;
    }
    *plan = p;
    return BLAZ_OK;
}

int blaz_batch_run(blaz_plan *plan, void *stream)
{
    if (!plan) return BLAZ_ERR_NULL;
    if (!plan->exec) return BLAZ_OK;
    cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? BLAZ_OK : set_cuda_error(e);
}

int blaz_batch_info_get(const blaz_plan *plan, blaz_batch_info *info)
{
    if (!plan || !info) return BLAZ_ERR_NULL;
    info->ops = (int64_t)plan->ops.size();
    info->items = plan->nitems;
    info->gemm_tiles = plan->ngemm;
    info->blocks_per_item = plan->cfg.blocks_per_item;
    info->ctas_per_sm = plan->cfg.ctas_per_sm;
    info->grid = plan->grid;
    info->scratch_bytes = (int64_t)(plan->scratch_bytes + plan->cap_items * sizeof(batch::Item) +
                                    plan->cap_partials * sizeof(double) + plan->ops.size() * sizeof(batch::DevOp));
    info->tuned_ms = plan->tuned_ms;
    return BLAZ_OK;
}

int blaz_batch_free(blaz_plan *plan)
{
    if (!plan) return BLAZ_ERR_NULL;
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    cudaFree(plan->d_ops);
    cudaFree(plan->d_items);
    cudaFree(plan->d_counters);
    cudaFree(plan->d_partials);
    cudaFree(plan->d_scratch);
    delete plan;
    return BLAZ_OK;
}

}  // extern "C"
