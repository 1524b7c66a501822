// Serving loop: continuous batching of mixed polymul / dot / GF(p^k) / matmul requests on one
// GPU.  A scheduler thread owns the device side:
//   admission   requests are taken in submission order; a batch reserves one block of the
//               device arena for all its inputs, descriptors and outputs, and waits while the
//               arena is full (admission by device memory);
//   batching    every admitted request waiting at a scheduler tick joins the next batch (up to
//               max_batch, or the pinned staging size), so requests that arrive while others
//               are on the GPU start in the next batch instead of waiting for a drain;
//   overlap     batches go round-robin to several CUDA streams, one batch in flight per
//               stream, so transfers and kernels of consecutive batches overlap;
//   per batch   one gathered host-to-device copy, one launch per request kind present (varlen
//               blocked-FQT polymul, segmented GF multiply per field, the persistent
//               matmul/dot kernel of the uneven batch), one device-to-host copy, an event;
//   completion  events are polled; results are scattered to the requests' host buffers and
//               the latency (submission to observed completion) is recorded.
// The GF(p^k) tables and the REDQ parameters stay resident in device memory across requests.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include <sys/prctl.h>

#include "arena.h"
#include "copy_pool.h"
#include "fpdqt_internal.cuh"

namespace fpd {

// ---- from k_batch.cu / k_gf.cu
fp_status batch_prepare(fp_ctx ctx, const fp_instance* in, size_t count, cudaStream_t st, bool measure_only,
                        std::vector<BInst>& insts, std::vector<BItem>& items);
size_t batch_plan_bytes(size_t ninst, size_t nitems);
void batch_plan_write(const std::vector<BInst>& insts, const std::vector<BItem>& items, uint8_t* h);
fp_status batch_launch_plan(fp_ctx ctx, size_t ninst, size_t nitems, uint8_t* d, cudaStream_t st);
fp_status gf_launch_segments(fp_ctx ctx, fp_gf g, uint8_t* base, const void* segs, uint32_t nseg, cudaStream_t st);
uint32_t gf_elem_bytes(fp_gf g);
uint32_t gf_order(fp_gf g);

// ---------------------------------------------------------------- varlen polymul kernel

struct PmDesc {
  uint64_t a, b, c;      // byte offsets from the batch base
  uint32_t ka, kb, d1, pad;
  RedqParams P;
};

__global__ void __launch_bounds__(256) k_polymul_var(uint8_t* base, const PmDesc* __restrict__ descs, uint32_t n,
                                                     uint32_t* err) {
  __shared__ uint64_t wa[1024];
  __shared__ uint64_t wb[1024];
  __shared__ uint8_t res[4096 + 64];
  __shared__ uint8_t ptab[1024];
  uint32_t bad = 0;
  for (uint32_t r = blockIdx.x; r < n; r += gridDim.x) {
    const PmDesc D = descs[r];
    __syncthreads();
    fill_pair_table(ptab, D.P);
    __syncthreads();
    Corrector C;
    C.init(D.P, ptab);
    fqt_block_product(base + D.a, base + D.b, base + D.c, D.ka, D.kb, D.d1, D.P, C, wa, wb, res, bad);
  }
  if (bad) flag_error(err, ERR_RANGE);
}

struct GfSegH { uint64_t a, b, c; uint32_t count, pad; };  // same layout as the device GfSeg

static inline double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
static inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
static inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace fpd

using namespace fpd;

struct fp_server_s {
  struct Req {
    fp_request r;
    uint64_t ticket;
    double t_submit;
    size_t in_a, in_b, out;   // byte sizes
    bool tc = false;          // matmul on the e4m3 tensor-core kernel (rows at 16-byte strides)
  };
  struct Batch {
    std::vector<Req> reqs;
    std::vector<size_t> out_off;   // per request, within the output region
    int stream;
    size_t blk_off, blk_bytes, out_region, out_bytes;
    cudaEvent_t ev;
  };
  fp_ctx ctx = nullptr;
  fp_server_config cfg{};
  uint8_t* arena = nullptr;
  FirstFitArena blocks;                           // free runs of the arena (first fit)
  std::vector<cudaStream_t> streams;
  std::vector<uint8_t*> h_in, h_out;              // pinned staging per stream
  size_t stage_bytes = 0;
  std::vector<int> stream_busy;
  std::vector<cudaEvent_t> events;
  std::mutex qmu;
  std::deque<Req> incoming;
  std::deque<Req> pending;
  std::deque<Batch> inflight;
  std::mutex rmu;
  std::vector<double> lat;                         // by ticket; -2 = not done, -1 = failed
  std::atomic<uint64_t> submitted{0}, completed{0}, batches{0}, launches{0}, failed{0};
  std::atomic<bool> stop{false};
  std::atomic<bool> force_stop{false};
  std::thread th;
  int device = 0;
  // gather / scatter copies of large batches spread over host threads (small batches stay on
  // the scheduler thread: waking the pool costs more than their copies)
  std::unique_ptr<CopyPool> pool;
  static constexpr size_t PARALLEL_COPY_BYTES = 256 << 10;

  void finish(Batch& b, bool ok) {
    const double t = now_s();
    if (ok) {
      auto scatter = [&](size_t i) {
        const Req& q = b.reqs[i];
        memcpy(q.r.host_out, h_out[b.stream] + b.out_off[i], q.out);
      };
      if (pool && b.out_bytes >= PARALLEL_COPY_BYTES) pool->run(b.reqs.size(), scatter);
      else for (size_t i = 0; i < b.reqs.size(); ++i) scatter(i);
    }
    {
      std::lock_guard<std::mutex> lk(rmu);
      for (const Req& q : b.reqs) lat[q.ticket] = ok ? (t - q.t_submit) * 1e6 : -1.0;
    }
    completed += b.reqs.size();
    if (!ok) failed += b.reqs.size();
    blocks.release(b.blk_off, b.blk_bytes);
    stream_busy[b.stream] = 0;
  }

  // Build and issue one batch from the front of `pending` on stream s.  Returns false if the
  // arena cannot hold even the first waiting request right now.
  bool launch_batch(int s) {
    // take requests while the whole batch block (inputs, descriptors, plan, outputs; laid out
    // exactly as below) fits one staging buffer, up to max_batch requests
    size_t in_bytes = 0, out_bytes = 0, npm = 0, nmm = 0, nitems = 0, nsegs = 0;
    std::vector<Req> take;
    std::unordered_map<fp_gf, uint32_t> nseg;
    while (!pending.empty() && take.size() < cfg.max_batch) {
      const Req& q = pending.front();
      const fp_request& r = q.r;
      size_t items_add = 0;
      if (r.kind == 1) items_add = 1;
      if (r.kind == 3 && !q.tc) {
        const bool pk = r.p <= 3 && r.c >= 448 && r.c <= 32767;
        const size_t nw = pk ? (r.b + 1) / 2 : r.b;
        items_add = ((r.a + 63) / 64) * ((nw + 63) / 64);
      }
      const size_t n_in = in_bytes + al16(q.in_a) + al16(q.in_b);
      const size_t n_pm = npm + (r.kind == 0), n_seg = nsegs + (r.kind == 2);
      const size_t n_mm = nmm + (r.kind == 1 || (r.kind == 3 && !q.tc)), n_it = nitems + items_add;
      const size_t block = al256(al256(al256(al256(n_in) + n_pm * sizeof(PmDesc)) + n_seg * sizeof(GfSegH)) +
                                 (n_mm ? batch_plan_bytes(n_mm, n_it) : 0)) +
                           out_bytes + al16(q.out);
      if (!take.empty() && block > stage_bytes) break;
      in_bytes = n_in;
      out_bytes += al16(q.out);
      npm = n_pm; nsegs = n_seg; nmm = n_mm; nitems = n_it;
      if (r.kind == 2) nseg[r.gf]++;
      take.push_back(q);
      pending.pop_front();
    }
    if (take.empty()) return false;
    // dot / matmul instances (device pointers are known once the block is placed)
    std::vector<fp_instance> mm;
    // block layout: [inputs | polymul descs | gf segs | batch plan | outputs]
    size_t off = 0;
    std::vector<size_t> ia(take.size()), ib(take.size());
    for (size_t i = 0; i < take.size(); ++i) {
      ia[i] = off; off += al16(take[i].in_a);
      ib[i] = off; off += al16(take[i].in_b);
    }
    const size_t pm_off = al256(off);
    off = pm_off + npm * sizeof(PmDesc);
    size_t seg_total = 0;
    for (auto& kv : nseg) seg_total += kv.second;
    const size_t seg_off = al256(off);
    off = seg_off + seg_total * sizeof(GfSegH);
    // batch plan size needs the item count: plan with a placeholder base first
    std::vector<BInst> insts;
    std::vector<BItem> items;
    const size_t plan_off = al256(off);
    // outputs
    std::vector<size_t> oo(take.size());
    // provisional: compute output offsets after the plan (plan size computed below)
    // fill instances with offsets relative to 0, fix up after placing
    for (size_t i = 0; i < take.size(); ++i) {
      const fp_request& r = take[i].r;
      if (r.kind == 1 || (r.kind == 3 && !take[i].tc)) {
        fp_instance x{};
        x.kind = r.kind == 1 ? 1u : 0u;
        x.p = r.p;
        if (r.kind == 1) { x.m = 1; x.n = 1; x.k = r.a; }
        else { x.m = r.a; x.n = r.b; x.k = r.c; }
        // fixed packing rule of the uneven batch (no timing inside the serving loop)
        x.reserved = (x.kind == 0 && r.p <= 3 && x.k >= 448 && x.k <= 32767) ? 1u : 0u;
        x.A = (const uint8_t*)(uintptr_t)(ia[i] + 1);   // non-null placeholders, fixed below
        x.B = (const uint8_t*)(uintptr_t)(ib[i] + 1);
        x.C = (uint8_t*)(uintptr_t)(i + 1);
        mm.push_back(x);
      }
    }
    size_t plan_bytes = 0;
    if (!mm.empty()) {
      if (batch_prepare(ctx, mm.data(), mm.size(), streams[s], true, insts, items) != FP_OK) {
        // invalid instances were rejected at submit; treat as failure of this batch
        Batch fb;
        fb.reqs = take;
        fb.stream = s;
        fb.blk_off = 0;
        fb.blk_bytes = 0;
        fb.out_off.assign(take.size(), 0);
        std::lock_guard<std::mutex> lk(rmu);
        for (const Req& q : take) lat[q.ticket] = -1.0;
        completed += take.size();
        failed += take.size();
        return true;
      }
      plan_bytes = batch_plan_bytes(insts.size(), items.size());
    }
    size_t out_region = al256(plan_off + plan_bytes);
    off = out_region;
    for (size_t i = 0; i < take.size(); ++i) { oo[i] = off - out_region; off += al16(take[i].out); }
    const size_t total = al256(off);
    // total <= stage_bytes by construction (the take loop above used this exact layout)
    size_t blk = 0;
    if (!blocks.alloc(total, &blk)) {
      for (auto it = take.rbegin(); it != take.rend(); ++it) pending.push_front(*it);
      return false;
    }
    uint8_t* dbase = arena + blk;
    uint8_t* hin = h_in[s];
    // gather inputs (tensor-core matmuls: operand rows at 16-byte strides)
    std::vector<fp_mm_problem> tcp;
    size_t gather_bytes = 0;
    for (size_t i = 0; i < take.size(); ++i) {
      const fp_request& r = take[i].r;
      gather_bytes += take[i].in_a + take[i].in_b;
      if (take[i].tc)
        tcp.push_back(fp_mm_problem{r.p, (int)r.a, (int)r.b, (int)r.c, nullptr, (int)al16(r.c), nullptr,
                                    (int)al16(r.b), nullptr, (int)r.b});
    }
    auto gather = [&](size_t i) {
      const fp_request& r = take[i].r;
      if (take[i].tc) {
        const size_t lda = al16(r.c), ldb = al16(r.b);
        const uint8_t* a = (const uint8_t*)r.host_a;
        const uint8_t* b = (const uint8_t*)r.host_b;
        for (uint32_t row = 0; row < r.a; ++row) memcpy(hin + ia[i] + row * lda, a + (size_t)row * r.c, r.c);
        for (uint32_t row = 0; row < r.c; ++row) memcpy(hin + ib[i] + row * ldb, b + (size_t)row * r.b, r.b);
        return;
      }
      memcpy(hin + ia[i], r.host_a, take[i].in_a);
      if (take[i].in_b) memcpy(hin + ib[i], r.host_b, take[i].in_b);
    };
    if (pool && gather_bytes >= PARALLEL_COPY_BYTES) pool->run(take.size(), gather);
    else for (size_t i = 0; i < take.size(); ++i) gather(i);
    // polymul descriptors
    PmDesc* pd = reinterpret_cast<PmDesc*>(hin + pm_off);
    uint32_t ipm = 0;
    for (size_t i = 0; i < take.size(); ++i) {
      const fp_request& r = take[i].r;
      if (r.kind != 0) continue;
      PmDesc D{};
      D.a = ia[i]; D.b = ib[i]; D.c = out_region + oo[i];
      D.ka = r.a + 1; D.kb = r.b + 1;
      uint32_t d1 = 1, bq = 1;
      fqt_params(r.p, D.ka, D.kb, &d1, &bq);
      D.d1 = d1;
      D.P = make_redq(r.p, bq, 2 * d1 - 1);
      pd[ipm++] = D;
    }
    // GF segments grouped by field
    GfSegH* sg = reinterpret_cast<GfSegH*>(hin + seg_off);
    std::vector<std::pair<fp_gf, std::pair<uint32_t, uint32_t>>> fields;  // field, (first, count)
    uint32_t iseg = 0;
    for (auto& kv : nseg) {
      uint32_t first = iseg;
      for (size_t i = 0; i < take.size(); ++i) {
        const fp_request& r = take[i].r;
        if (r.kind != 2 || r.gf != kv.first) continue;
        sg[iseg++] = GfSegH{ia[i], ib[i], out_region + oo[i], r.a, 0};
      }
      fields.push_back({kv.first, {first, iseg - first}});
    }
    // dot / matmul plan with real device pointers
    if (!mm.empty()) {
      size_t j = 0;
      for (size_t i = 0; i < take.size(); ++i) {
        const fp_request& r = take[i].r;
        if (r.kind != 1 && (r.kind != 3 || take[i].tc)) continue;
        mm[j].A = dbase + ia[i];
        mm[j].B = dbase + ib[i];
        mm[j].C = dbase + out_region + oo[i];
        ++j;
      }
      insts.clear();
      items.clear();
      batch_prepare(ctx, mm.data(), mm.size(), streams[s], true, insts, items);
      batch_plan_write(insts, items, hin + plan_off);
    }
    cudaStream_t st = streams[s];
    bool ok = cudaMemcpyAsync(dbase, hin, out_region, cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok && npm) {
      const int grid = (int)std::min<size_t>(npm, (size_t)ctx->num_sms * 4);
      FP_LAUNCH(ctx, "k_polymul_var", st,
                k_polymul_var<<<grid, 256, 0, st>>>(dbase, (const PmDesc*)(dbase + pm_off), (uint32_t)npm, ctx->d_err));
      ok = cudaGetLastError() == cudaSuccess;
      launches++;
    }
    for (auto& f : fields) {
      if (!ok) break;
      ok = gf_launch_segments(ctx, f.first, dbase, dbase + seg_off + (size_t)f.second.first * sizeof(GfSegH),
                              f.second.second, st) == FP_OK;
      launches++;
    }
    if (ok && !mm.empty()) {
      ok = batch_launch_plan(ctx, insts.size(), items.size(), dbase + plan_off, st) == FP_OK;
      launches++;
    }
    if (ok && !tcp.empty()) {
      // the e4m3 kernel's grouped launches (it range-checks its operands itself; parameters only,
      // no context scratch, so the serving thread may call it)
      std::vector<const fp_mm_problem*> ptr;
      size_t j = 0;
      for (size_t i = 0; i < take.size(); ++i) {
        if (!take[i].tc) continue;
        tcp[j].A = dbase + ia[i];
        tcp[j].B = dbase + ib[i];
        tcp[j].C = dbase + out_region + oo[i];
        ptr.push_back(&tcp[j]);
        ++j;
      }
      ok = launch_mm_f8_grouped_locked(ctx, ptr.data(), ptr.size(), st) == FP_OK;
      launches += (ptr.size() + FP_GROUP_MAX - 1) / FP_GROUP_MAX;
    }
    if (ok) ok = cudaMemcpyAsync(h_out[s], dbase + out_region, total - out_region, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    Batch b;
    b.reqs = std::move(take);
    b.out_off = oo;
    b.stream = s;
    b.blk_off = blk;
    b.blk_bytes = total;
    b.out_region = out_region;
    b.out_bytes = total - out_region;
    b.ev = events[s];
    if (ok) ok = cudaEventRecord(b.ev, st) == cudaSuccess;
    batches++;
    stream_busy[s] = 1;
    if (!ok) {
      cudaStreamSynchronize(st);
      finish(b, false);
      return true;
    }
    inflight.push_back(std::move(b));
    return true;
  }

  void loop() {
    cudaSetDevice(device);
    // the idle wait below is a few microseconds: with the default 50 us timer slack every idle
    // iteration would sleep ~55 us, late both for new requests and for completed batches
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
    double oldest_wait_start = 0;
    while (true) {
      {
        std::lock_guard<std::mutex> lk(qmu);
        while (!incoming.empty()) {
          pending.push_back(incoming.front());
          incoming.pop_front();
        }
      }
      bool progressed = false;
      // completions (any order)
      for (auto it = inflight.begin(); it != inflight.end();) {
        cudaError_t e = cudaEventQuery(it->ev);
        if (e == cudaErrorNotReady) { ++it; continue; }
        finish(*it, e == cudaSuccess);
        it = inflight.erase(it);
        progressed = true;
      }
      // launches: while a stream is free and requests wait
      if (!pending.empty()) {
        if (oldest_wait_start == 0) oldest_wait_start = now_s();
        const bool gpu_busy = !inflight.empty();
        const bool window_open = gpu_busy && pending.size() < cfg.max_batch &&
                                 (now_s() - pending.front().t_submit) * 1e6 < cfg.window_us;
        if (!window_open) {
          for (int s = 0; s < (int)streams.size() && !pending.empty(); ++s) {
            if (stream_busy[s]) continue;
            if (!launch_batch(s)) break;   // arena full: wait for completions
            progressed = true;
          }
        }
      } else {
        oldest_wait_start = 0;
      }
      if (force_stop) break;
      if (stop && pending.empty() && inflight.empty()) {
        std::lock_guard<std::mutex> lk(qmu);
        if (incoming.empty()) break;
      }
      if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(2));
    }
  }
};

extern "C" fp_status fp_server_create(fp_ctx ctx, const fp_server_config* cfg, fp_server* out) {
  FP_CHECK(ctx && cfg && out, FP_EINVAL, "fp_server_create: null argument");
  FP_CHECK(cfg->streams >= 1 && cfg->streams <= 16, FP_EINVAL, "fp_server_create: streams in [1, 16]");
  FP_CHECK(cfg->arena_bytes >= (1u << 20), FP_EINVAL, "fp_server_create: arena must be >= 1 MiB");
  FP_CHECK(cfg->max_batch >= 1, FP_EINVAL, "fp_server_create: max_batch must be >= 1");
  *out = nullptr;
  fp_server s = new (std::nothrow) fp_server_s();
  FP_CHECK(s != nullptr, FP_ENOMEM, "fp_server_create: out of host memory");
  s->ctx = ctx;
  s->cfg = *cfg;
  s->device = ctx->device;
  const cudaError_t de = cudaSetDevice(ctx->device);
  if (de != cudaSuccess) {
    delete s;
    return cuda_fail(de, "fp_server_create: cudaSetDevice");
  }
  cudaError_t e = cudaMalloc(&s->arena, cfg->arena_bytes);
  if (e != cudaSuccess) { delete s; set_error("fp_server_create: arena of %llu bytes", (unsigned long long)cfg->arena_bytes); return FP_ENOMEM; }
  s->blocks.reset(cfg->arena_bytes);
  s->stage_bytes = std::min<size_t>(cfg->arena_bytes / cfg->streams, (size_t)256 << 20);
  // every resource is recorded as soon as it exists, so that fp_server_destroy frees a
  // partly built server (its scheduler thread has not started yet)
  auto fail = [s]() {
    fp_server_destroy(s);
    set_error("fp_server_create: stream / pinned staging allocation failed");
    return FP_ENOMEM;
  };
  for (uint32_t i = 0; i < cfg->streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail();
    s->streams.push_back(st);
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail();
    s->events.push_back(ev);
    uint8_t* hi;
    if (cudaMallocHost(&hi, s->stage_bytes) != cudaSuccess) return fail();
    s->h_in.push_back(hi);
    uint8_t* ho;
    if (cudaMallocHost(&ho, s->stage_bytes) != cudaSuccess) return fail();
    s->h_out.push_back(ho);
    s->stream_busy.push_back(0);
  }
  {
    // copy workers: the host's cores less three (the submitting thread, the scheduler, the rest
    // of the process), at most 7
    const int hc = (int)std::thread::hardware_concurrency();
    const int nw = std::max(0, std::min(7, hc - 3));
    if (nw > 0) s->pool.reset(new (std::nothrow) CopyPool(nw));
  }
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return FP_OK;
}

// Validates one request and fills its queue entry (sizes, tensor-core route); nothing queued.
static fp_status server_prepare(fp_server s, const fp_request* r, fp_server_s::Req& q) {
  FP_CHECK(r->host_a && r->host_out, FP_EINVAL, "fp_server_submit: null host buffer");
  q = fp_server_s::Req{};
  q.r = *r;
  switch (r->kind) {
    case 0:
      FP_CHECK(r->p >= 2 && r->p <= 251 && is_prime(r->p), FP_EINVAL, "polymul request: p=%u", r->p);
      FP_CHECK(r->a <= 1023 && r->b <= 1023 && r->host_b, FP_EINVAL, "polymul request: degrees <= 1023");
      q.in_a = r->a + 1; q.in_b = r->b + 1; q.out = (size_t)r->a + r->b + 1;
      {
        uint32_t d1, bq;
        FP_CHECK(fqt_params(r->p, r->a + 1, r->b + 1, &d1, &bq), FP_EBOUND, "polymul request: no FQT packing");
      }
      break;
    case 1:
      FP_CHECK(r->p >= 2 && r->p <= 251 && is_prime(r->p), FP_EINVAL, "dot request: p=%u", r->p);
      FP_CHECK(r->a >= 1 && r->host_b, FP_EINVAL, "dot request: empty");
      q.in_a = r->a; q.in_b = r->a; q.out = 4;
      break;
    case 2:
      FP_CHECK(r->gf != nullptr && r->a >= 1 && r->host_b, FP_EINVAL, "GF request: field / count");
      q.in_a = q.in_b = q.out = (size_t)r->a * gf_elem_bytes(r->gf);
      break;
    case 3:
      FP_CHECK(r->p >= 2 && r->p <= 251 && is_prime(r->p), FP_EINVAL, "matmul request: p=%u", r->p);
      FP_CHECK(r->a >= 1 && r->b >= 1 && r->c >= 1 && r->host_b, FP_EINVAL, "matmul request: sizes");
      FP_CHECK((uint64_t)r->c * (r->p - 1) * (r->p - 1) < (1ull << 32), FP_EBOUND, "matmul request: k (p-1)^2");
      q.in_a = (size_t)r->a * r->c; q.in_b = (size_t)r->c * r->b; q.out = (size_t)r->a * r->b;
      // large products with exact e4m3 residues go to the tensor cores, rows padded to 16 bytes
      q.tc = r->p <= 17 && r->a >= 64 && r->b >= 64 && (uint64_t)r->c * (r->p - 1) * (r->p - 1) < (1ull << 24) &&
             (uint64_t)r->a * r->b * r->c >= (1ull << 21) && r->a <= (1u << 20) && r->b <= (1u << 20) &&
             r->c <= (1u << 20);
      if (q.tc) { q.in_a = (size_t)r->a * al16(r->c); q.in_b = (size_t)r->c * al16(r->b); }
      break;
    default:
      FP_CHECK(false, FP_EINVAL, "request kind %u", r->kind);
  }
  FP_CHECK(al16(q.in_a) + al16(q.in_b) + al16(q.out) + (1u << 20) <= s->stage_bytes, FP_EINVAL,
           "request larger than the staging area (%zu bytes)", s->stage_bytes);
  return FP_OK;
}

// Queues prepared requests with consecutive tickets (one lock of each queue for all of them).
static uint64_t server_enqueue(fp_server s, std::vector<fp_server_s::Req>& qs) {
  uint64_t first;
  {
    std::lock_guard<std::mutex> lk(s->rmu);
    first = s->lat.size();
    s->lat.resize(first + qs.size(), -2.0);
  }
  const double t = now_s();
  for (size_t i = 0; i < qs.size(); ++i) {
    qs[i].ticket = first + i;
    qs[i].t_submit = t;
  }
  {
    std::lock_guard<std::mutex> lk(s->qmu);
    for (auto& q : qs) s->incoming.push_back(q);
  }
  s->submitted += qs.size();
  return first;
}

extern "C" fp_status fp_server_submit(fp_server s, const fp_request* r, uint64_t* ticket) {
  FP_CHECK(s && r && ticket, FP_EINVAL, "fp_server_submit: null argument");
  std::vector<fp_server_s::Req> qs(1);
  fp_status st = server_prepare(s, r, qs[0]);
  if (st != FP_OK) return st;
  *ticket = server_enqueue(s, qs);
  return FP_OK;
}

extern "C" fp_status fp_server_submit_many(fp_server s, const fp_request* reqs, size_t n, uint64_t* first_ticket) {
  FP_CHECK(s && first_ticket && (reqs || n == 0), FP_EINVAL, "fp_server_submit_many: null argument");
  std::vector<fp_server_s::Req> qs(n);
  for (size_t i = 0; i < n; ++i) {
    fp_status st = server_prepare(s, &reqs[i], qs[i]);
    if (st != FP_OK) return st;
  }
  *first_ticket = server_enqueue(s, qs);
  return FP_OK;
}

extern "C" fp_status fp_server_poll(fp_server s, uint64_t ticket, int* done, double* latency_us) {
  FP_CHECK(s && done, FP_EINVAL, "fp_server_poll: null argument");
  std::lock_guard<std::mutex> lk(s->rmu);
  FP_CHECK(ticket < s->lat.size(), FP_EINVAL, "fp_server_poll: unknown ticket");
  double l = s->lat[ticket];
  *done = l == -2.0 ? 0 : (l == -1.0 ? -1 : 1);
  if (latency_us) *latency_us = l;
  return FP_OK;
}

extern "C" fp_status fp_server_drain(fp_server s, double timeout_s) {
  FP_CHECK(s != nullptr, FP_EINVAL, "fp_server_drain: null server");
  const double t0 = now_s();
  while (s->completed.load() < s->submitted.load()) {
    if (now_s() - t0 > timeout_s) {
      set_error("fp_server_drain: %llu of %llu requests done after %.1f s",
                (unsigned long long)s->completed.load(), (unsigned long long)s->submitted.load(), timeout_s);
      return FP_ETIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  return FP_OK;
}

extern "C" fp_status fp_server_latencies(fp_server s, uint64_t first, size_t n, double* out) {
  FP_CHECK(s && out, FP_EINVAL, "fp_server_latencies: null argument");
  std::lock_guard<std::mutex> lk(s->rmu);
  for (size_t i = 0; i < n; ++i) {
    const uint64_t t = first + i;
    out[i] = t < s->lat.size() && s->lat[t] >= 0 ? s->lat[t] : -1.0;
  }
  return FP_OK;
}

extern "C" fp_status fp_server_stats_get(fp_server s, fp_server_stats* out) {
  FP_CHECK(s && out, FP_EINVAL, "fp_server_stats_get: null argument");
  out->submitted = s->submitted.load();
  out->completed = s->completed.load();
  out->batches = s->batches.load();
  out->launches = s->launches.load();
  out->failed = s->failed.load();
  return FP_OK;
}

extern "C" void fp_server_destroy(fp_server s) {
  if (!s) return;
  if (s->th.joinable()) {
    if (fp_server_drain(s, 60.0) != FP_OK) s->force_stop = true;
    s->stop = true;
    s->th.join();
  }
  cudaSetDevice(s->device);
  for (auto st : s->streams) cudaStreamSynchronize(st);
  for (auto st : s->streams) cudaStreamDestroy(st);
  for (auto e : s->events) cudaEventDestroy(e);
  for (auto p : s->h_in) cudaFreeHost(p);
  for (auto p : s->h_out) cudaFreeHost(p);
  if (s->arena) cudaFree(s->arena);
  delete s;
}
