// Serving runtime: continuous batching of evaluation requests on one GPU.
//
// A request is a population (genome tensors in the Section 3.1 encoding), a
// batch of input vectors per genome and a number of steps; step s evaluates
// the population on observations generated on the device from
// (request seed, s).  The server owns one device pool of `hbm_budget_bytes`
// (allocated once) and a scheduler thread:
//   admission  queued requests take pool memory first-fit, in arrival order
//              (a later request that fits may pass one that does not); the
//              genome tensors are copied in and transformed (Section 3.3,
//              transformation stage, once per request);
//   ticks      every tick advances each active request by one step: one
//              kernel fills all their observations, one launch of the
//              persistent multi-population kernel evaluates all of them
//              (each request one bucket, at its own step);
//   completion a request whose last step's tick has finished on the GPU is
//              stamped done, its pool memory returns, waiters wake.
// Requests that arrive while others run join at the next tick: their work
// overlaps on the device with the requests already active.  A genome's
// outputs do not depend on what else shares its launch, so each request's
// results are identical alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "neat_device.cuh"
#include "neat_internal.h"
#include "neat_trace.h"

namespace neat {
namespace {

// ---- Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds of the
// Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and a Weyl key
// schedule 0x9E3779B9 / 0xBB67AE85, written from that definition.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = U4{(uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0, 1) from the top 24 bits.
__device__ __forceinline__ float unit_open(uint32_t b) { return ((float)(b >> 8) + 0.5f) * (1.0f / 16777216.0f); }

// Elements 4b .. 4b+3 of (seed, step): standard normals by Box-Muller on
// Philox block b (counter = (b low, b high, step, 0x4f4253)): words (x, y)
// give elements 4b (cos) and 4b+1 (sin), words (z, w) elements 4b+2, 4b+3.
__device__ __forceinline__ void normals_of_block(uint64_t seed, int step, uint64_t blk, float out[4])
{
    const U4 r = philox4x32_10(U4{(uint32_t)blk, (uint32_t)(blk >> 32), (uint32_t)step, 0x4f4253u}, (uint32_t)seed,
                               (uint32_t)(seed >> 32));
    float s, c;
    const float rad0 = sqrtf(-2.0f * logf(unit_open(r.x)));
    sincospif(2.0f * unit_open(r.y), &s, &c);
    out[0] = rad0 * c;
    out[1] = rad0 * s;
    const float rad1 = sqrtf(-2.0f * logf(unit_open(r.z)));
    sincospif(2.0f * unit_open(r.w), &s, &c);
    out[2] = rad1 * c;
    out[3] = rad1 * s;
}

struct GenDesc {
    float *out;
    uint64_t count;
    uint64_t seed;
    int step;
    int block_begin;   // first block of this descriptor
};

constexpr int kGenThreads = 256;
constexpr int kGenPerBlock = kGenThreads * 4;

__global__ void gen_normals_kernel(const GenDesc *__restrict__ descs, int nd)
{
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (descs[mid].block_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const GenDesc d = descs[lo];
    const uint64_t e0 = (uint64_t)(blockIdx.x - d.block_begin) * kGenPerBlock + 4u * threadIdx.x;
    if (e0 >= d.count) return;
    float z[4];
    normals_of_block(d.seed, d.step, e0 >> 2, z);
    for (int k = 0; k < 4 && e0 + k < d.count; ++k) d.out[e0 + k] = z[k];
}

// One descriptor, passed by value.
__global__ void fill_normals_kernel(float *out, uint64_t count, uint64_t seed, int step)
{
    const uint64_t e0 = ((uint64_t)blockIdx.x * kGenThreads + threadIdx.x) * 4u;
    if (e0 >= count) return;
    float z[4];
    normals_of_block(seed, step, e0 >> 2, z);
    for (int k = 0; k < 4 && e0 + k < count; ++k) out[e0 + k] = z[k];
}

// Raw Philox words: word e = component e mod 4 of the block for counter
// (e / 4 low, e / 4 high, stream low, stream high ^ 0x574f5244), key = seed.
__global__ void gen_words_kernel(uint32_t *out, uint64_t n, uint64_t seed, uint64_t stream)
{
    const uint64_t blocks = (n + 3) >> 2;
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < blocks;
         b += (uint64_t)gridDim.x * blockDim.x) {
        const U4 r = philox4x32_10(U4{(uint32_t)b, (uint32_t)(b >> 32), (uint32_t)stream,
                                      (uint32_t)(stream >> 32) ^ 0x574f5244u},
                                   (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint64_t e = b << 2;
        if (e + 3 < n) {
            out[e] = r.x; out[e + 1] = r.y; out[e + 2] = r.z; out[e + 3] = r.w;
        } else {
            const uint32_t v[4] = {r.x, r.y, r.z, r.w};
            for (uint64_t k = 0; e + k < n; ++k) out[e + k] = v[k];
        }
    }
}

__global__ void fill_identity(int32_t *idx, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) idx[i] = i;
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) of the device pool, 256-byte granules.
class PoolAllocator {
  public:
    explicit PoolAllocator(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

enum ReqState { kQueued, kActive, kDone };

struct Request {
    uint64_t ticket = 0;
    neat_request r{};
    std::vector<float> nodes, conns;    // host copies taken at submit
    double t_submit = 0, t_admit = -1, t_done = -1;
    ReqState state = kQueued;
    int status = NEAT_EAGAIN;
    bool cancel = false;
    size_t off = 0, bytes = 0;          // pool block
    size_t o_nodes = 0, o_conns = 0, o_rec = 0, o_obs = 0, o_status = 0;
    int next_step = 0;
    long last_tick = -1;                // last tick this request took part in
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t request_bytes(const neat_request &r, size_t *o_nodes, size_t *o_conns, size_t *o_rec, size_t *o_obs,
                     size_t *o_status)
{
    size_t off = 0;
    *o_nodes = off;
    off += align256((size_t)r.pop * r.dims.max_nodes * 5 * 4);
    *o_conns = off;
    off += align256((size_t)r.pop * std::max(r.dims.max_conns, 1) * 4 * 4);
    *o_rec = off;
    off += align256(record_stride(r.dims) * (size_t)r.pop);
    *o_obs = off;
    off += align256((size_t)r.pop * r.batch * std::max(r.dims.num_inputs, 1) * 4);
    *o_status = off;
    off += align256((size_t)r.pop * 4);
    return off;
}

}  // namespace
}  // namespace neat

using namespace neat;

struct neat_server {
    neat_serve_cfg cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    unsigned char *pool = nullptr;
    std::unique_ptr<PoolAllocator> alloc;
    // device tables of one tick
    BucketDev *d_buckets = nullptr;
    GenDesc *d_gen = nullptr;
    unsigned int *d_counter = nullptr;
    int32_t *d_identity = nullptr;
    // persistent block of a tick: 1024 threads lets the tile rows of large
    // requests' genomes (up to 16 threads per row) share a block with others;
    // on the serving workload it cut p99 latency from 11.9 to 8.6 ms against
    // 256 threads
    int block_threads = 1024;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::string worker_error;

    // ticks in flight: (tick id, event)
    std::deque<std::pair<long, cudaEvent_t>> inflight;
    std::vector<cudaEvent_t> event_pool;
    long next_tick = 0, done_tick = -1;
    double busy_ms = 0;
    long ticks = 0;
};

namespace neat {
namespace {

cudaEvent_t take_event(neat_server *S)
{
    if (!S->event_pool.empty()) {
        cudaEvent_t e = S->event_pool.back();
        S->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

// Retire finished ticks; complete the requests whose last tick is done.
void retire(neat_server *S, bool block_oldest)
{
    while (!S->inflight.empty()) {
        auto &f = S->inflight.front();
        cudaError_t q = block_oldest ? cudaEventSynchronize(f.second) : cudaEventQuery(f.second);
        if (q == cudaErrorNotReady) break;
        block_oldest = false;
        S->done_tick = f.first;
        S->event_pool.push_back(f.second);
        S->inflight.pop_front();
    }
    std::lock_guard<std::mutex> lk(S->mu);
    const double t = now_ms();
    bool any = false;
    for (auto &kv : S->reqs) {
        Request &R = *kv.second;
        if (R.state != kActive || R.last_tick > S->done_tick) continue;
        const bool finished = R.next_step >= R.r.steps;
        if (!finished && !R.cancel) continue;
        R.state = kDone;
        R.t_done = t;
        R.status = R.cancel && !finished ? NEAT_ECANCELLED : NEAT_OK;
        S->alloc->release(R.off, R.bytes);
        std::vector<float>().swap(R.nodes);
        std::vector<float>().swap(R.conns);
        any = true;
    }
    if (any) {
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

void worker_main(neat_server *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<Request *> admitted, active;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            auto has_work = [&] {
                if (S->stop || !S->inflight.empty()) return true;
                for (auto &kv : S->reqs)
                    if (kv.second->state == kActive) return true;
                for (uint64_t t : S->queue) {
                    Request &R = *S->reqs[t];
                    size_t a, b, c, d, e;
                    if (request_bytes(R.r, &a, &b, &c, &d, &e) <= S->cfg.hbm_budget_bytes - S->alloc->used()) return true;
                }
                return false;
            };
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5), has_work);
            if (S->stop && S->inflight.empty()) {
                bool busy = false;
                for (auto &kv : S->reqs) busy |= kv.second->state == kActive;
                if (!busy) break;
            }
            // admission: arrival order, a later request may pass one that does not fit
            int active_n = 0;
            for (auto &kv : S->reqs) active_n += kv.second->state == kActive;
            for (auto it = S->queue.begin(); it != S->queue.end() && active_n < S->cfg.max_active;) {
                Request &R = *S->reqs[*it];
                if (R.cancel) {
                    R.state = kDone;
                    R.status = NEAT_ECANCELLED;
                    R.t_done = now_ms();
                    it = S->queue.erase(it);
                    S->cv_done.notify_all();
                    continue;
                }
                R.bytes = request_bytes(R.r, &R.o_nodes, &R.o_conns, &R.o_rec, &R.o_obs, &R.o_status);
                if (S->alloc->alloc(R.bytes, &R.off)) {
                    R.state = kActive;
                    R.t_admit = now_ms();
                    admitted.push_back(&R);
                    ++active_n;
                    it = S->queue.erase(it);
                } else {
                    ++it;
                }
            }
            for (auto &kv : S->reqs) {
                Request &R = *kv.second;
                if (R.state == kActive && !R.cancel && R.next_step < R.r.steps) active.push_back(&R);
            }
        }
        cudaError_t e = cudaSuccess;
        for (Request *R : admitted) {
            unsigned char *base = S->pool + R->off;
            const neat_request &r = R->r;
            const bool borrow = (r.flags & NEAT_REQ_BORROW_HOST) != 0;
            const float *hn = borrow ? r.nodes_host : R->nodes.data();
            const float *hc = borrow ? r.conns_host : R->conns.data();
            const size_t nn = (size_t)r.pop * r.dims.max_nodes * 5, nc = (size_t)r.pop * r.dims.max_conns * 4;
            e = cudaMemcpyAsync(base + R->o_nodes, hn, nn * 4, cudaMemcpyHostToDevice, S->stream);
            if (e == cudaSuccess && nc)
                e = cudaMemcpyAsync(base + R->o_conns, hc, nc * 4, cudaMemcpyHostToDevice, S->stream);
            int rc = neat_transform(reinterpret_cast<float *>(base + R->o_nodes),
                                    reinterpret_cast<float *>(base + R->o_conns), r.pop, r.dims, base + R->o_rec,
                                    record_stride(r.dims) * (size_t)r.pop,
                                    reinterpret_cast<uint32_t *>(base + R->o_status), S->stream);
            if (rc != NEAT_OK || e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->worker_error = neat_last_error();
            }
        }
        if (!active.empty()) {
            TraceRange trace_range("neat_serve_tick");
            const long tick = S->next_tick++;
            std::vector<GenDesc> gen;
            std::vector<BucketDev> table;
            size_t smem_regions = 0;
            int blocks = 0, items = 0;
            for (Request *R : active) {
                unsigned char *base = S->pool + R->off;
                const neat_request &r = R->r;
                const uint64_t count = (uint64_t)r.pop * r.batch * r.dims.num_inputs;
                if (count) {
                    gen.push_back(GenDesc{reinterpret_cast<float *>(base + R->o_obs), count, r.obs_seed, R->next_step,
                                          blocks});
                    blocks += (int)((count + kGenPerBlock - 1) / kGenPerBlock);
                }
                neat_pop_desc pd;
                pd.transformed_dev = base + R->o_rec;
                pd.pop = r.pop;
                pd.dims = r.dims;
                pd.batch = r.batch;
                pd.inputs_dev = reinterpret_cast<const float *>(base + R->o_obs);
                pd.in_step_stride = 0;
                pd.outputs_dev = r.outputs_dev + (size_t)R->next_step * r.out_step_stride;
                pd.out_step_stride = 0;
                BucketDev b;
                size_t fp = 0;
                if (fill_population_bucket(pd, S->d_identity, S->block_threads, items, &b, &fp) == NEAT_OK) {
                    table.push_back(b);
                    items += b.cta_items;
                    smem_regions = std::max(smem_regions, fp);
                }
                R->next_step++;
                R->last_tick = tick;
            }
            if (!gen.empty() && blocks > 0) {
                e = cudaMemcpyAsync(S->d_gen, gen.data(), gen.size() * sizeof(GenDesc), cudaMemcpyHostToDevice,
                                    S->stream);
                gen_normals_kernel<<<blocks, kGenThreads, 0, S->stream>>>(S->d_gen, (int)gen.size());
            }
            e = cudaMemcpyAsync(S->d_buckets, table.data(), table.size() * sizeof(BucketDev), cudaMemcpyHostToDevice,
                                S->stream);
            cudaMemsetAsync(S->d_counter, 0, sizeof(unsigned int), S->stream);
            const int rc = launch_plan_table(S->d_buckets, (int)table.size(), items, S->d_counter, 0, smem_regions,
                                             S->block_threads, S->stream);
            if (rc != NEAT_OK) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->worker_error = neat_last_error();
            }
            cudaEvent_t ev = take_event(S);
            cudaEventRecord(ev, S->stream);
            S->inflight.emplace_back(tick, ev);
            S->ticks++;
        }
        retire(S, S->inflight.size() > 2);
    }
    while (!S->inflight.empty()) retire(S, true);
}

}  // namespace
}  // namespace neat

extern "C" int neat_serve_create(const neat_serve_cfg *cfg, neat_server **out)
{
    clear_error();
    if (!cfg || !out) return invalid("neat_serve_create: null pointer");
    *out = nullptr;
    if (cfg->hbm_budget_bytes < (1u << 20)) return invalid("neat_serve_create: budget below 1 MiB");
    if (cfg->max_active < 1 || cfg->max_active > 4096) return invalid("neat_serve_create: max_active in 1..4096");
    neat_server *S = new neat_server();
    S->cfg = *cfg;
    cudaGetDevice(&S->device);
    cudaError_t e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&S->pool, cfg->hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_buckets, sizeof(BucketDev) * (size_t)cfg->max_active);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_gen, sizeof(GenDesc) * (size_t)cfg->max_active);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_identity, sizeof(int32_t) * 65536);
    if (e != cudaSuccess) {
        neat_serve_destroy(S);
        return e == cudaErrorMemoryAllocation ? (set_error("neat_serve_create: out of device memory"), NEAT_ENOMEM)
                                              : cuda_fail(e, "neat_serve_create");
    }
    fill_identity<<<64, 256, 0, S->stream>>>(S->d_identity, 65536);
    cudaStreamSynchronize(S->stream);
    S->alloc.reset(new PoolAllocator(cfg->hbm_budget_bytes));
    S->worker = std::thread(worker_main, S);
    *out = S;
    return NEAT_OK;
}

extern "C" int neat_serve_submit(neat_server *S, const neat_request *r, uint64_t *ticket)
{
    clear_error();
    if (!S || !r || !ticket) return invalid("neat_serve_submit: null pointer");
    if (!dims_ok(r->dims)) return invalid("neat_serve_submit: invalid dims");
    if (r->pop < 1 || r->pop > 65536 || r->batch < 1 || r->steps < 1)
        return invalid("neat_serve_submit: pop in 1..65536, batch and steps >= 1");
    if (!r->nodes_host || (r->dims.max_conns > 0 && !r->conns_host) || !r->outputs_dev)
        return invalid("neat_serve_submit: null genome or output pointer");
    std::unique_ptr<Request> R(new Request());
    R->r = *r;
    size_t a, b, c, d, e;
    if (request_bytes(R->r, &a, &b, &c, &d, &e) > S->cfg.hbm_budget_bytes) {
        set_error("neat_serve_submit: the request can never fit the server's memory budget");
        return NEAT_EBUDGET;
    }
    {
        neat_pop_desc pd{};
        pd.pop = r->pop;
        pd.dims = r->dims;
        pd.batch = r->batch;
        BucketDev tmp;
        size_t fp;
        if (fill_population_bucket(pd, nullptr, S->block_threads, 0, &tmp, &fp) != NEAT_OK) return NEAT_EINVAL;
    }
    if (!(r->flags & NEAT_REQ_BORROW_HOST)) {
        R->nodes.assign(r->nodes_host, r->nodes_host + (size_t)r->pop * r->dims.max_nodes * 5);
        R->conns.assign(r->conns_host ? r->conns_host : r->nodes_host,
                        (r->conns_host ? r->conns_host : r->nodes_host) + (size_t)r->pop * r->dims.max_conns * 4);
    }
    R->t_submit = now_ms();
    std::lock_guard<std::mutex> lk(S->mu);
    R->ticket = S->next_ticket++;
    *ticket = R->ticket;
    S->queue.push_back(R->ticket);
    S->reqs[R->ticket] = std::move(R);
    S->cv_work.notify_all();
    return NEAT_OK;
}

static void fill_result(const Request &R, neat_result *res)
{
    res->status = R.status;
    res->submit_ms = R.t_submit;
    res->admit_ms = R.t_admit;
    res->done_ms = R.t_done;
    res->genome_forwards = (uint64_t)R.r.pop * R.r.batch * (uint64_t)std::min(R.next_step, R.r.steps);
}

extern "C" int neat_serve_poll(neat_server *S, uint64_t ticket, neat_result *res)
{
    clear_error();
    if (!S || !res) return invalid("neat_serve_poll: null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return invalid("neat_serve_poll: unknown ticket");
    if (it->second->state != kDone) return NEAT_EAGAIN;
    fill_result(*it->second, res);
    return it->second->status;
}

extern "C" int neat_serve_wait(neat_server *S, uint64_t ticket, int32_t timeout_ms, neat_result *res)
{
    clear_error();
    if (!S || !res) return invalid("neat_serve_wait: null pointer");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return invalid("neat_serve_wait: unknown ticket");
    Request *R = it->second.get();
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(timeout_ms, 0)),
                                        [&] { return R->state == kDone; });
    if (!ok) {
        set_error("neat_serve_wait: timed out");
        return NEAT_ETIMEOUT;
    }
    fill_result(*R, res);
    return R->status;
}

extern "C" int neat_serve_cancel(neat_server *S, uint64_t ticket)
{
    clear_error();
    if (!S) return invalid("neat_serve_cancel: null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return invalid("neat_serve_cancel: unknown ticket");
    it->second->cancel = true;
    S->cv_work.notify_all();
    return NEAT_OK;
}

extern "C" int neat_serve_stats(neat_server *S, neat_serve_report *st)
{
    clear_error();
    if (!S || !st) return invalid("neat_serve_stats: null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> lat, wait;
    double first = 1e300, last = 0;
    uint64_t gf = 0;
    int queued = 0, active = 0, done = 0, cancelled = 0;
    for (auto &kv : S->reqs) {
        const Request &R = *kv.second;
        if (R.state == kQueued) ++queued;
        if (R.state == kActive) ++active;
        if (R.state != kDone) continue;
        if (R.status != NEAT_OK) {
            ++cancelled;
            continue;
        }
        ++done;
        lat.push_back(R.t_done - R.t_submit);
        wait.push_back(R.t_admit - R.t_submit);
        first = std::min(first, R.t_submit);
        last = std::max(last, R.t_done);
        gf += (uint64_t)R.r.pop * R.r.batch * (uint64_t)R.r.steps;
    }
    auto pct = [](std::vector<double> v, double p) {
        if (v.empty()) return 0.0;
        std::sort(v.begin(), v.end());
        const size_t i = std::min(v.size() - 1, (size_t)std::ceil(p * (double)v.size()) - (p > 0 ? 1 : 0));
        return v[i];
    };
    st->completed = done;
    st->cancelled = cancelled;
    st->queued = queued;
    st->active = active;
    st->latency_p50_ms = pct(lat, 0.50);
    st->latency_p99_ms = pct(lat, 0.99);
    st->queue_wait_p50_ms = pct(wait, 0.50);
    st->queue_wait_p99_ms = pct(wait, 0.99);
    st->genome_forwards = gf;
    st->genome_forwards_per_s = (done && last > first) ? (double)gf / ((last - first) / 1e3) : 0.0;
    st->ticks = S->ticks;
    st->pool_used_bytes = S->alloc ? S->alloc->used() : 0;
    return NEAT_OK;
}

extern "C" void neat_serve_destroy(neat_server *S)
{
    if (!S) return;
    if (S->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
            for (uint64_t t : S->queue) S->reqs[t]->cancel = true;
            for (auto &kv : S->reqs) kv.second->cancel = true;
        }
        S->cv_work.notify_all();
        S->worker.join();
    }
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (auto &f : S->inflight) cudaEventDestroy(f.second);
    for (cudaEvent_t ev : S->event_pool) cudaEventDestroy(ev);
    if (S->pool) cudaFree(S->pool);
    if (S->d_buckets) cudaFree(S->d_buckets);
    if (S->d_gen) cudaFree(S->d_gen);
    if (S->d_counter) cudaFree(S->d_counter);
    if (S->d_identity) cudaFree(S->d_identity);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

extern "C" int neat_fill_normal(uint64_t seed, int32_t step, int64_t count, float *out_dev, void *stream)
{
    clear_error();
    if (count < 0 || step < 0) return invalid("neat_fill_normal: negative size or step");
    if (count == 0) return NEAT_OK;
    if (!out_dev) return invalid("neat_fill_normal: null pointer");
    const long blocks = (count + kGenPerBlock - 1) / kGenPerBlock;
    if (blocks > 0x7fffffffL) return invalid("neat_fill_normal: count too large");
    fill_normals_kernel<<<(unsigned)blocks, kGenThreads, 0, as_stream(stream)>>>(out_dev, (uint64_t)count, seed, step);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_fill_normal: launch");
    return NEAT_OK;
}

extern "C" int neat_fill_words(uint64_t seed, uint64_t stream, uint32_t *words_dev, int64_t n, void *s)
{
    clear_error();
    if (n < 0) return invalid("neat_fill_words: n < 0");
    if (n == 0) return NEAT_OK;
    if (!words_dev) return invalid("neat_fill_words: null pointer");
    const uint64_t blocks = ((uint64_t)n + 3) / 4;
    const unsigned grid = (unsigned)std::min<uint64_t>((blocks + 255) / 256, 152u * 16u);
    gen_words_kernel<<<grid, 256, 0, as_stream(s)>>>(words_dev, (uint64_t)n, seed, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neat_fill_words: launch");
    return NEAT_OK;
}
