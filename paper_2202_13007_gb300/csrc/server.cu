// server.cu -- request server over the compressed-matrix kernels: resident
// compressed matrices, admission by device memory, continuous batching.
//
// Requests (the operations of Sec. III of "Compressed Matrix Computations",
// arXiv 2202.13007, on resident compressed matrices) are queued by any host
// thread.  A scheduler thread:
//   1. completes in-flight launches whose event has fired (copies results to
//      the callers' buffers, marks new resident matrices ready, returns their
//      working memory to the budget);
//   2. when a stream slot is free, admits queued requests in arrival order
//      whose operands are ready and whose memory fits the budget, up to
//      max_batch, and launches them as one persistent batch (batch kernel);
//   3. waits at most max_wait_us for more requests when a launch is already
//      in flight, so that batches grow under load and stay small when idle.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_internal.cuh"

namespace blaz {
namespace srv {

using Clock = std::chrono::steady_clock;

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
static int64_t nblocks(int64_t r, int64_t c) { return (r / 8) * (c / 8); }
static size_t cmat_bytes(int64_t r, int64_t c)
{
    const int64_t nb = nblocks(r, c);
    return up256(8 * nb) * 2 + up256((size_t)kKeep * nb) + up256(nb);
}

// Pinned host staging buffers, reused by size class (power of two >= 4 KiB).
class PinnedPool {
  public:
    ~PinnedPool()
    {
        for (auto &kv : free_)
            for (void *p : kv.second) cudaFreeHost(p);
    }
    void *get(size_t bytes, size_t &cls)
    {
        cls = 4096;
        while (cls < bytes) cls <<= 1;
        std::lock_guard<std::mutex> lk(mu_);
        auto &v = free_[cls];
        if (!v.empty()) {
            void *p = v.back();
            v.pop_back();
            return p;
        }
        void *p = nullptr;
        if (cudaHostAlloc(&p, cls, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void put(void *p, size_t cls)
    {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        free_[cls].push_back(p);
    }

  private:
    std::mutex mu_;
    std::map<size_t, std::vector<void *>> free_;
};

struct Resident {
    blaz_cmat m{};
    void *base = nullptr;
    size_t bytes = 0;
    bool ready = false;      // producing launch completed
    int refs = 0;            // submitted, unfinished requests reading it
    bool releasing = false;  // a RELEASE is queued
};

struct Ticket {
    uint64_t id = 0;
    blaz_request req{};
    Clock::time_point t_submit, t_done;
    int status = 1;          // 1 pending
    uint64_t handle = 0;     // output handle (allocated at submit)
    double value = 0.0;
    void *in_stage = nullptr;  // pinned copy of host_A or host_B (or the caller's pinned buffer)
    size_t in_cls = 0, in_bytes = 0;
    int64_t in_rows = 0, in_cols = 0, in_ld = 0;  // host layout of in_stage
    bool pinned = false;       // BLAZ_REQ_PINNED: no staging copies
    size_t need = 0;         // working bytes while in flight (excludes the resident output)
    size_t out_res_bytes = 0;
};

struct Launch {
    int slot = -1;
    std::vector<Ticket *> tickets;
    void *work = nullptr;    // device working memory of the launch
    size_t work_bytes = 0;
    void *out_stage = nullptr;
    size_t out_cls = 0;
    std::vector<size_t> out_off;  // offset of each ticket's output in out_stage
    std::vector<size_t> split_off; // split-bf16 products: decompressed operand and slice scratch
    void *desc_stage = nullptr;
    size_t desc_cls = 0;
    cudaEvent_t done = nullptr;
};

}  // namespace srv
}  // namespace blaz

using namespace blaz;
using namespace blaz::srv;

struct blaz_server {
    blaz_server_cfg cfg{};
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::vector<Launch *> inflight;
    PinnedPool pinned;  // declared before the streams are destroyed: freed last

    std::mutex mu;                  // guards everything below
    std::condition_variable cv_submit, cv_done;
    std::deque<Ticket *> queue;     // submitted, not yet admitted
    std::unordered_map<uint64_t, Ticket *> tickets;
    std::unordered_map<uint64_t, Resident> residents;
    uint64_t next_ticket = 1, next_handle = 1;
    size_t used_bytes = 0, peak_bytes = 0;  // resident + in-flight working memory
    bool stop = false;
    std::thread worker;

    // statistics
    int64_t submitted = 0, completed = 0, rejected = 0, launches = 0, batched = 0;
    std::vector<double> latencies;
    Clock::time_point first_submit, last_done;
    bool any_submit = false;
};

namespace {

// Device bytes a request needs while in flight, and the bytes of the resident
// matrix it creates.
int request_needs(blaz_server *s, const blaz_request &r, size_t &need, size_t &out_res, int64_t &orows,
                  int64_t &ocols)
{
    need = 0;
    out_res = 0;
    orows = ocols = 0;
    auto res = [&](uint64_t h, Resident *&o) -> int {
        auto it = s->residents.find(h);
        if (it == s->residents.end() || it->second.releasing) return BLAZ_ERR_ARG;
        o = &it->second;
        return BLAZ_OK;
    };
    Resident *a = nullptr, *b = nullptr;
    switch (r.kind) {
    case BLAZ_OP_COMPRESS:
        if (r.rows < 0 || r.cols < 0 || r.rows % 8 || r.cols % 8) return BLAZ_ERR_SHAPE;
        if (nblocks(r.rows, r.cols) && !r.host_A) return BLAZ_ERR_NULL;
        if (nblocks(r.rows, r.cols) && r.lda < r.cols) return BLAZ_ERR_LD;
        need = up256((size_t)(r.rows * r.cols) * 8);
        out_res = cmat_bytes(r.rows, r.cols);
        orows = r.rows;
        ocols = r.cols;
        return BLAZ_OK;
    case BLAZ_OP_DECOMPRESS:
        if (res(r.a, a)) return BLAZ_ERR_ARG;
        if (!r.host_out) return BLAZ_ERR_NULL;
        if (r.ldo < a->m.cols) return BLAZ_ERR_LD;
        need = up256((size_t)(a->m.rows * a->m.cols) * 8);
        return BLAZ_OK;
    case BLAZ_OP_ADD:
    case BLAZ_OP_SUB:
    case BLAZ_OP_DOT:
        if (res(r.a, a) || res(r.b, b)) return BLAZ_ERR_ARG;
        if (a->m.rows != b->m.rows || a->m.cols != b->m.cols) return BLAZ_ERR_SHAPE;
        if (r.kind == BLAZ_OP_DOT) {
            if (!r.host_out) return BLAZ_ERR_NULL;
            need = 256;
        } else {
            out_res = cmat_bytes(a->m.rows, a->m.cols);
            orows = a->m.rows;
            ocols = a->m.cols;
        }
        return BLAZ_OK;
    case BLAZ_OP_SCALE:
        if (res(r.a, a)) return BLAZ_ERR_ARG;
        out_res = cmat_bytes(a->m.rows, a->m.cols);
        orows = a->m.rows;
        ocols = a->m.cols;
        return BLAZ_OK;
    case BLAZ_OP_MATMUL: {
        if (res(r.a, a)) return BLAZ_ERR_ARG;
        if (r.m < 0) return BLAZ_ERR_SHAPE;
        const int64_t n = a->m.rows, k = a->m.cols;
        if (n && r.m && (!r.host_out || (k && !r.host_B))) return BLAZ_ERR_NULL;
        if (n && r.m && (r.ldo < r.m || (k && r.ldb < r.m))) return BLAZ_ERR_LD;
        need = up256((size_t)(k * r.m) * 8) + up256((size_t)(n * r.m) * 8) + up256((size_t)(n * k) * 8);
        if (s->cfg.matmul_mode == BLAZ_MM_SPLIT_BF16) need += up256(split_bf16_scratch_bytes(n, k, r.m));
        return BLAZ_OK;
    }
    case BLAZ_REQ_RELEASE:
        if (res(r.a, a)) return BLAZ_ERR_ARG;
        return BLAZ_OK;
    default:
        return BLAZ_ERR_ARG;
    }
}

void finish_ticket(blaz_server *s, Ticket *t, int status)
{
    t->status = status;
    t->t_done = Clock::now();
    if (t->in_stage && !t->pinned) s->pinned.put(t->in_stage, t->in_cls);
    t->in_stage = nullptr;
    if (status == BLAZ_OK) {
        s->completed++;
        s->latencies.push_back(std::chrono::duration<double, std::micro>(t->t_done - t->t_submit).count());
        s->last_done = t->t_done;
    } else {
        s->rejected++;
    }
}

// Operand handles of a request (0 when unused).
void operands(const blaz_request &r, uint64_t &a, uint64_t &b)
{
    a = b = 0;
    switch (r.kind) {
    case BLAZ_OP_ADD:
    case BLAZ_OP_SUB:
    case BLAZ_OP_DOT: a = r.a; b = r.b; break;
    case BLAZ_OP_DECOMPRESS:
    case BLAZ_OP_SCALE:
    case BLAZ_OP_MATMUL:
    case BLAZ_REQ_RELEASE: a = r.a; break;
    default: break;
    }
}

// Complete a launch whose event fired (scheduler thread, lock held).
void complete_launch(blaz_server *s, Launch *L)
{
    for (size_t i = 0; i < L->tickets.size(); ++i) {
        Ticket *t = L->tickets[i];
        const blaz_request &r = t->req;
        const char *out = (const char *)L->out_stage + L->out_off[i];
        if (r.kind == BLAZ_OP_DOT) {
            if (t->pinned) {
                t->value = *r.host_out;
            } else {
                std::memcpy(&t->value, out, sizeof(double));
                if (r.host_out) *r.host_out = t->value;
            }
        } else if ((r.kind == BLAZ_OP_DECOMPRESS || r.kind == BLAZ_OP_MATMUL) && !t->pinned) {
            const blaz_cmat &a = s->residents[r.a].m;
            const int64_t rows = a.rows, cols = r.kind == BLAZ_OP_MATMUL ? r.m : a.cols;
            for (int64_t q = 0; q < rows; ++q)
                std::memcpy(r.host_out + q * r.ldo, out + (size_t)q * cols * 8, (size_t)cols * 8);
        }
        if (t->handle) s->residents[t->handle].ready = true;
        uint64_t ha, hb;
        operands(r, ha, hb);
        if (ha) s->residents[ha].refs--;
        if (hb) s->residents[hb].refs--;
        s->used_bytes -= t->need;
        finish_ticket(s, t, BLAZ_OK);
    }
    cudaFreeAsync(L->work, s->streams[L->slot]);
    s->pinned.put(L->out_stage, L->out_cls);
    s->pinned.put(L->desc_stage, L->desc_cls);
    cudaEventDestroy(L->done);
    s->slot_busy[L->slot] = false;
    delete L;
    s->cv_done.notify_all();
}

// Launch the admitted tickets on a free slot (scheduler thread, lock held).
int launch_impl(blaz_server *s, int slot, std::vector<Ticket *> &adm, Launch *L);

int launch(blaz_server *s, int slot, std::vector<Ticket *> &adm)
{
    Launch *L = new Launch();
    int rc = launch_impl(s, slot, adm, L);
    if (rc) {  // nothing of L is in flight when launch_impl fails before its last enqueue
        cudaStreamSynchronize(s->streams[slot]);
        if (L->work) cudaFreeAsync(L->work, s->streams[slot]);
        s->pinned.put(L->out_stage, L->out_cls);
        s->pinned.put(L->desc_stage, L->desc_cls);
        if (L->done) cudaEventDestroy(L->done);
        delete L;
    }
    return rc;
}

int launch_impl(blaz_server *s, int slot, std::vector<Ticket *> &adm, Launch *L)
{
    cudaStream_t st = s->streams[slot];
    L->slot = slot;
    L->tickets = adm;
    // Working memory layout: per ticket inputs / outputs, then batch arrays.
    std::vector<size_t> in_off(adm.size(), 0), dev_out_off(adm.size(), 0);
    size_t work = 0, out_host = 0;
    L->out_off.assign(adm.size(), 0);
    for (size_t i = 0; i < adm.size(); ++i) {
        const blaz_request &r = adm[i]->req;
        if (r.kind == BLAZ_OP_COMPRESS || r.kind == BLAZ_OP_MATMUL) {
            in_off[i] = work;
            work += up256(adm[i]->in_bytes);
        }
        size_t ob = 0;
        if (r.kind == BLAZ_OP_DOT) ob = 8;
        if (r.kind == BLAZ_OP_DECOMPRESS) ob = (size_t)(s->residents[r.a].m.rows * s->residents[r.a].m.cols) * 8;
        if (r.kind == BLAZ_OP_MATMUL) ob = (size_t)(s->residents[r.a].m.rows * r.m) * 8;
        dev_out_off[i] = work;
        work += up256(ob);
        L->out_off[i] = out_host;
        if (!adm[i]->pinned) out_host += up256(ob);
    }
    // Split-bf16 products: decompressed operand + slices, after the batch launch.
    const bool split = s->cfg.matmul_mode == BLAZ_MM_SPLIT_BF16;
    L->split_off.assign(adm.size(), 0);
    if (split)
        for (size_t i = 0; i < adm.size(); ++i)
            if (adm[i]->req.kind == BLAZ_OP_MATMUL) {
                const blaz_cmat &a = s->residents[adm[i]->req.a].m;
                L->split_off[i] = work;
                work += up256((size_t)(a.rows * a.cols) * 8) + up256(split_bf16_scratch_bytes(a.rows, a.cols, adm[i]->req.m));
            }
    // Resident outputs: allocate their storage now.
    std::vector<blaz_op> ops;
    ops.reserve(adm.size());
    for (size_t i = 0; i < adm.size(); ++i) {
        Ticket *t = adm[i];
        const blaz_request &r = t->req;
        if (t->handle) {
            Resident &R = s->residents[t->handle];
            cudaError_t ea = cudaMallocAsync(&R.base, R.bytes ? R.bytes : 256, st);
            if (ea != cudaSuccess) {
                R.base = nullptr;
                cudaGetLastError();
                return ea == cudaErrorMemoryAllocation ? BLAZ_ERR_OOM : set_cuda_error(ea);
            }
            const int64_t nb = nblocks(R.m.rows, R.m.cols);
            char *b = (char *)R.base;
            R.m.f = (double *)b;
            R.m.s = (double *)(b + up256(8 * nb));
            R.m.code = (int8_t *)(b + 2 * up256(8 * nb));
            R.m.phi = (uint8_t *)(b + 2 * up256(8 * nb) + up256((size_t)kKeep * nb));
        }
        (void)r;
    }
    // Batch descriptors (sized after the ops are known).
    for (size_t i = 0; i < adm.size(); ++i) {
        Ticket *t = adm[i];
        const blaz_request &r = t->req;
        blaz_op o;
        std::memset(&o, 0, sizeof(o));
        o.kind = r.kind;
        if (r.kind == BLAZ_OP_COMPRESS) {
            o.out = s->residents[t->handle].m;
            o.lda = r.cols;
        } else {
            o.a = s->residents[r.a].m;
            if (r.kind == BLAZ_OP_ADD || r.kind == BLAZ_OP_SUB || r.kind == BLAZ_OP_DOT) o.b = s->residents[r.b].m;
            if (t->handle) o.out = s->residents[t->handle].m;
            o.c = r.c;
            o.m = r.m;
            o.ldb = r.m;
            o.ldc = r.kind == BLAZ_OP_MATMUL ? r.m : o.a.cols;
        }
        ops.push_back(o);
    }
    std::vector<batch::DevOp> dops;
    std::vector<batch::Item> items;
    int64_t partials = 0;
    size_t scratch = 0;
    int ngemm = 0;
    const int64_t bpi = 128;
    batch::build_work(ops.data(), (int)ops.size(), bpi, nullptr, dops, items, partials, scratch, ngemm);
    const size_t off_scratch = work;
    work += up256(scratch);
    const size_t off_ops = work;
    work += up256(sizeof(batch::DevOp) * std::max<size_t>(1, dops.size()));
    const size_t off_items = work;
    work += up256(sizeof(batch::Item) * std::max<size_t>(1, items.size()));
    const size_t off_cnt = work;
    work += up256(sizeof(unsigned) * (1 + ops.size()));
    const size_t off_part = work;
    work += up256(sizeof(double) * std::max<int64_t>(1, partials));
    L->work_bytes = work;
    cudaError_t e = cudaMallocAsync(&L->work, work, st);
    if (e != cudaSuccess) {
        L->work = nullptr;
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? BLAZ_ERR_OOM : set_cuda_error(e);
    }
    char *W = (char *)L->work;
    // Device pointers of inputs and outputs, then the final descriptors.
    for (size_t i = 0; i < adm.size(); ++i) {
        const blaz_request &r = adm[i]->req;
        if (r.kind == BLAZ_OP_COMPRESS) ops[i].A = (const double *)(W + in_off[i]);
        if (r.kind == BLAZ_OP_MATMUL) ops[i].B = (const double *)(W + in_off[i]);
        if (r.kind == BLAZ_OP_DOT) ops[i].result = (double *)(W + dev_out_off[i]);
        if (r.kind == BLAZ_OP_DECOMPRESS || r.kind == BLAZ_OP_MATMUL) ops[i].C = (double *)(W + dev_out_off[i]);
    }
    if (split)
        for (size_t i = 0; i < adm.size(); ++i)
            if (adm[i]->req.kind == BLAZ_OP_MATMUL) {
                ops[i].kind = BLAZ_OP_DECOMPRESS;
                ops[i].C = (double *)(W + L->split_off[i]);
                ops[i].ldc = ops[i].a.cols;
            }
    batch::build_work(ops.data(), (int)ops.size(), bpi, W + off_scratch, dops, items, partials, scratch, ngemm);
    const size_t desc_bytes = sizeof(batch::DevOp) * dops.size() + sizeof(batch::Item) * items.size();
    L->desc_stage = s->pinned.get(std::max<size_t>(desc_bytes, 1), L->desc_cls);
    L->out_stage = s->pinned.get(std::max<size_t>(out_host, 1), L->out_cls);
    if (!L->desc_stage || !L->out_stage) return BLAZ_ERR_OOM;
    std::memcpy(L->desc_stage, dops.data(), sizeof(batch::DevOp) * dops.size());
    std::memcpy((char *)L->desc_stage + sizeof(batch::DevOp) * dops.size(), items.data(),
                sizeof(batch::Item) * items.size());
    // Host -> device: inputs, descriptors; zero the counters.
    for (size_t i = 0; i < adm.size(); ++i) {
        const Ticket *t = adm[i];
        if (t->in_stage && t->in_bytes)
            cudaMemcpy2DAsync(W + in_off[i], (size_t)t->in_cols * 8, t->in_stage, (size_t)t->in_ld * 8,
                              (size_t)t->in_cols * 8, (size_t)t->in_rows, cudaMemcpyHostToDevice, st);
    }
    if (!dops.empty())
        cudaMemcpyAsync(W + off_ops, L->desc_stage, sizeof(batch::DevOp) * dops.size(), cudaMemcpyHostToDevice, st);
    if (!items.empty())
        cudaMemcpyAsync(W + off_items, (char *)L->desc_stage + sizeof(batch::DevOp) * dops.size(),
                        sizeof(batch::Item) * items.size(), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(W + off_cnt, 0, sizeof(unsigned) * (1 + ops.size()), st);
    const int grid = std::max(1, std::min<int>(num_sms() * 2, (int)items.size()));
    int rc = batch::launch((batch::DevOp *)(W + off_ops), (batch::Item *)(W + off_items), (int)items.size(),
                           (unsigned *)(W + off_cnt), (double *)(W + off_part), grid, st);
    if (rc) return rc;
    if (split)
        for (size_t i = 0; i < adm.size(); ++i)
            if (adm[i]->req.kind == BLAZ_OP_MATMUL) {
                const blaz_request &r = adm[i]->req;
                const int64_t n = ops[i].a.rows, k = ops[i].a.cols;
                double *Ah = (double *)(W + L->split_off[i]);
                char *sl = W + L->split_off[i] + up256((size_t)(n * k) * 8);
                if ((rc = launch_matmul_split_bf16(Ah, k, (const double *)(W + in_off[i]), r.m,
                                                   (double *)(W + dev_out_off[i]), r.m, n, k, r.m, sl, st)))
                    return rc;
            }
    // Device -> host: results.
    for (size_t i = 0; i < adm.size(); ++i) {
        const blaz_request &r = adm[i]->req;
        size_t ob = 0;
        if (r.kind == BLAZ_OP_DOT) ob = 8;
        if (r.kind == BLAZ_OP_DECOMPRESS) ob = (size_t)(ops[i].a.rows * ops[i].a.cols) * 8;
        if (r.kind == BLAZ_OP_MATMUL) ob = (size_t)(ops[i].a.rows * r.m) * 8;
        if (!ob) continue;
        if (adm[i]->pinned) {
            const int64_t rows = r.kind == BLAZ_OP_DOT ? 1 : ops[i].a.rows;
            const int64_t cols = r.kind == BLAZ_OP_DOT ? 1 : (r.kind == BLAZ_OP_MATMUL ? r.m : ops[i].a.cols);
            const int64_t ldo = r.kind == BLAZ_OP_DOT ? 1 : r.ldo;
            cudaMemcpy2DAsync(r.host_out, (size_t)ldo * 8, W + dev_out_off[i], (size_t)cols * 8, (size_t)cols * 8,
                              (size_t)rows, cudaMemcpyDeviceToHost, st);
        } else {
            cudaMemcpyAsync((char *)L->out_stage + L->out_off[i], W + dev_out_off[i], ob, cudaMemcpyDeviceToHost, st);
        }
    }
    cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
    cudaEventRecord(L->done, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error(e);
    s->inflight.push_back(L);
    s->slot_busy[slot] = true;
    s->launches++;
    s->batched += (int64_t)adm.size();
    return BLAZ_OK;
}

void scheduler(blaz_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // 1. completions
        for (size_t i = 0; i < s->inflight.size();) {
            Launch *L = s->inflight[i];
            cudaError_t q = cudaEventQuery(L->done);
            if (q == cudaSuccess) {
                s->inflight.erase(s->inflight.begin() + i);
                complete_launch(s, L);
            } else {
                if (q != cudaErrorNotReady) cudaGetLastError();
                ++i;
            }
        }
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;
        // 2. releases whose matrix is idle
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Ticket *t = *it;
            if (t->req.kind == BLAZ_REQ_RELEASE) {
                auto r = s->residents.find(t->req.a);
                if (r != s->residents.end() && r->second.ready && r->second.refs == 0) {
                    if (r->second.base) cudaFreeAsync(r->second.base, s->streams[0]);
                    s->used_bytes -= r->second.bytes;
                    s->residents.erase(r);
                    finish_ticket(s, t, BLAZ_OK);
                    it = s->queue.erase(it);
                    s->cv_done.notify_all();
                    continue;
                }
            }
            ++it;
        }
        // 3. admission into a free slot
        int slot = -1;
        for (int q = 0; q < (int)s->slot_busy.size(); ++q)
            if (!s->slot_busy[q]) {
                slot = q;
                break;
            }
        bool launched = false;
        if (slot >= 0 && !s->queue.empty()) {
            const auto age = std::chrono::duration<double, std::micro>(Clock::now() - s->queue.front()->t_submit).count();
            const bool go = s->inflight.empty() || (int)s->queue.size() >= s->cfg.max_batch || age >= s->cfg.max_wait_us;
            if (go) {
                std::vector<Ticket *> adm;
                for (auto it = s->queue.begin(); it != s->queue.end() && (int)adm.size() < s->cfg.max_batch;) {
                    Ticket *t = *it;
                    const blaz_request &r = t->req;
                    if (r.kind == BLAZ_REQ_RELEASE) {
                        ++it;
                        continue;
                    }
                    uint64_t ha, hb;
                    operands(r, ha, hb);
                    auto ready = [&](uint64_t h) {
                        if (!h) return true;
                        auto f = s->residents.find(h);
                        return f != s->residents.end() && f->second.ready;
                    };
                    const bool gone = (ha && !s->residents.count(ha)) || (hb && !s->residents.count(hb));
                    if (gone) {  // operand released meanwhile
                        finish_ticket(s, t, BLAZ_ERR_ARG);
                        it = s->queue.erase(it);
                        s->cv_done.notify_all();
                        continue;
                    }
                    const size_t total = t->need + t->out_res_bytes;
                    if (ready(ha) && ready(hb) && s->used_bytes + total <= (size_t)s->cfg.budget_bytes) {
                        s->used_bytes += total;
                        s->peak_bytes = std::max(s->peak_bytes, s->used_bytes);
                        adm.push_back(t);
                        it = s->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                if (!adm.empty()) {
                    int rc = launch(s, slot, adm);
                    if (rc) {  // could not launch: fail these requests, return their memory
                        for (Ticket *t : adm) {
                            uint64_t ha, hb;
                            operands(t->req, ha, hb);
                            if (ha) s->residents[ha].refs--;
                            if (hb) s->residents[hb].refs--;
                            s->used_bytes -= t->need + t->out_res_bytes;
                            if (t->handle) {
                                Resident &R = s->residents[t->handle];
                                if (R.base) cudaFreeAsync(R.base, s->streams[slot]);
                                s->residents.erase(t->handle);
                            }
                            finish_ticket(s, t, rc);
                        }
                        s->cv_done.notify_all();
                    }
                    launched = true;
                }
            }
        }
        if (!launched) {
            // Sleep briefly: new submissions wake us, completions are polled.
            s->cv_submit.wait_for(lk, std::chrono::microseconds(s->inflight.empty() ? 200 : 10));
        }
    }
}

}  // namespace

extern "C" {

int blaz_server_create(const blaz_server_cfg *cfg, blaz_server **out)
{
    if (!cfg || !out) return BLAZ_ERR_NULL;
    if (cfg->budget_bytes <= 0 || cfg->streams < 0 || cfg->max_batch < 0 || cfg->max_wait_us < 0 ||
        cfg->queue_capacity < 0 || (cfg->matmul_mode != BLAZ_MM_FP64 && cfg->matmul_mode != BLAZ_MM_SPLIT_BF16))
        return BLAZ_ERR_ARG;
    blaz_server *s = new blaz_server();
    s->cfg = *cfg;
    if (s->cfg.streams == 0) s->cfg.streams = 4;
    if (s->cfg.max_batch == 0) s->cfg.max_batch = 512;
    if (s->cfg.max_wait_us == 0) s->cfg.max_wait_us = 100;
    if (s->cfg.queue_capacity == 0) s->cfg.queue_capacity = 65536;
    cudaGetDevice(&s->device);
    num_sms();
    for (int i = 0; i < s->cfg.streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return set_cuda_error(cudaGetLastError());
        }
        s->streams.push_back(st);
    }
    s->slot_busy.assign(s->cfg.streams, false);
    s->worker = std::thread(scheduler, s);
    *out = s;
    return BLAZ_OK;
}

int blaz_server_submit(blaz_server *s, const blaz_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket) return BLAZ_ERR_NULL;
    Ticket *t = new Ticket();
    t->req = *req;
    t->t_submit = Clock::now();
    // Copy the host inputs into pinned staging outside the lock.
    const blaz_request &r = *req;
    int64_t rows = 0, cols = 0, ld = 0;
    const double *src = nullptr;
    if (r.kind == BLAZ_OP_COMPRESS) {
        rows = r.rows;
        cols = r.cols;
        ld = r.lda;
        src = r.host_A;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        size_t need, outres;
        int64_t orows, ocols;
        int rc = request_needs(s, r, need, outres, orows, ocols);
        if (rc == BLAZ_OK && need + outres > (size_t)s->cfg.budget_bytes) rc = BLAZ_ERR_BUDGET;
        if (rc == BLAZ_OK && (int64_t)s->queue.size() >= s->cfg.queue_capacity) rc = BLAZ_ERR_BUSY;
        if (rc != BLAZ_OK) {
            if (rc != BLAZ_ERR_BUSY) s->rejected++;
            delete t;
            return rc;
        }
        t->need = need;
        t->out_res_bytes = outres;
        uint64_t ha, hb;
        operands(r, ha, hb);
        if (r.kind == BLAZ_REQ_RELEASE) {
            s->residents[ha].releasing = true;
        } else {
            if (ha) s->residents[ha].refs++;
            if (hb) s->residents[hb].refs++;
        }
        if (r.kind == BLAZ_OP_MATMUL) {
            rows = s->residents[r.a].m.cols;
            cols = r.m;
            ld = r.ldb;
            src = r.host_B;
        }
        if (outres) {  // reserve the handle of the new resident matrix now
            t->handle = s->next_handle++;
            Resident R;
            R.m.rows = orows;
            R.m.cols = ocols;
            R.bytes = outres;
            s->residents[t->handle] = R;
        }
    }
    t->pinned = (r.flags & BLAZ_REQ_PINNED) != 0;
    if (src && rows * cols > 0 && t->pinned) {
        t->in_bytes = (size_t)(rows * cols) * 8;
        t->in_stage = const_cast<double *>(src);
        t->in_rows = rows;
        t->in_cols = cols;
        t->in_ld = ld;
    } else if (src && rows * cols > 0) {
        t->in_bytes = (size_t)(rows * cols) * 8;
        t->in_rows = rows;
        t->in_cols = cols;
        t->in_ld = cols;
        t->in_stage = s->pinned.get(t->in_bytes, t->in_cls);
        if (!t->in_stage) {
            std::lock_guard<std::mutex> lk(s->mu);
            if (t->handle) s->residents.erase(t->handle);
            uint64_t ha, hb;
            operands(r, ha, hb);
            if (ha && s->residents.count(ha)) s->residents[ha].refs--;
            if (hb && s->residents.count(hb)) s->residents[hb].refs--;
            delete t;
            return BLAZ_ERR_OOM;
        }
        for (int64_t q = 0; q < rows; ++q)
            std::memcpy((char *)t->in_stage + (size_t)q * cols * 8, src + q * ld, (size_t)cols * 8);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        t->id = s->next_ticket++;
        s->tickets[t->id] = t;
        s->queue.push_back(t);
        s->submitted++;
        if (!s->any_submit) {
            s->any_submit = true;
            s->first_submit = t->t_submit;
        }
        *ticket = t->id;
    }
    s->cv_submit.notify_one();
    return BLAZ_OK;
}

static void fill_result(Ticket *t, blaz_result *res)
{
    res->status = t->status;
    res->handle = t->status == BLAZ_OK ? t->handle : 0;
    res->value = t->value;
    res->latency_us = t->status == 1 ? 0.0 : std::chrono::duration<double, std::micro>(t->t_done - t->t_submit).count();
}

int blaz_server_poll(blaz_server *s, uint64_t ticket, blaz_result *res)
{
    if (!s || !res) return BLAZ_ERR_NULL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return BLAZ_ERR_ARG;
    fill_result(it->second, res);
    if (it->second->status != 1) {
        delete it->second;
        s->tickets.erase(it);
    }
    return BLAZ_OK;
}

int blaz_server_wait(blaz_server *s, uint64_t ticket, blaz_result *res, int64_t timeout_us)
{
    if (!s || !res) return BLAZ_ERR_NULL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto deadline = Clock::now() + std::chrono::microseconds(timeout_us);
    while (true) {
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return BLAZ_ERR_ARG;
        if (it->second->status != 1) {
            fill_result(it->second, res);
            delete it->second;
            s->tickets.erase(it);
            return BLAZ_OK;
        }
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && Clock::now() >= deadline) {
            fill_result(it->second, res);
            return BLAZ_ERR_TIMEOUT;
        }
    }
}

int blaz_server_cmat(blaz_server *s, uint64_t handle, blaz_cmat *out)
{
    if (!s || !out) return BLAZ_ERR_NULL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->residents.find(handle);
    if (it == s->residents.end() || !it->second.ready) return BLAZ_ERR_ARG;
    *out = it->second.m;
    return BLAZ_OK;
}

int blaz_server_stats_get(blaz_server *s, blaz_server_stats *st)
{
    if (!s || !st) return BLAZ_ERR_NULL;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->launches = s->launches;
    st->resident_matrices = 0;
    st->resident_bytes = 0;
    for (auto &kv : s->residents)
        if (kv.second.ready) {
            st->resident_matrices++;
            st->resident_bytes += (int64_t)kv.second.bytes;
        }
    st->peak_bytes = (int64_t)s->peak_bytes;
    std::vector<double> v = s->latencies;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        st->p50_us = v[(size_t)(0.50 * (v.size() - 1))];
        st->p99_us = v[(size_t)(0.99 * (v.size() - 1))];
    } else {
        st->p50_us = st->p99_us = 0.0;
    }
    st->mean_batch = s->launches ? (double)s->batched / (double)s->launches : 0.0;
    const double span = s->completed ? std::chrono::duration<double>(s->last_done - s->first_submit).count() : 0.0;
    st->throughput_rps = span > 0 ? s->completed / span : 0.0;
    return BLAZ_OK;
}

int blaz_server_destroy(blaz_server *s)
{
    if (!s) return BLAZ_ERR_NULL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // Requests still waiting for memory or operands are cancelled.
        for (Ticket *t : s->queue) {
            if (t->req.kind != BLAZ_REQ_RELEASE) {
                if (t->handle) s->residents.erase(t->handle);
                finish_ticket(s, t, BLAZ_ERR_BUSY);
            } else {
                finish_ticket(s, t, BLAZ_ERR_BUSY);
            }
        }
        s->queue.clear();
    }
    s->cv_submit.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (auto &kv : s->residents)
        if (kv.second.base) cudaFreeAsync(kv.second.base, s->streams[0]);
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto &kv : s->tickets) delete kv.second;
    delete s;
    return BLAZ_OK;
}

}  // extern "C"
