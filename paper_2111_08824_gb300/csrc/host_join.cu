// join_host: the whole join from host buffers, pipelined in chunks.
//
// Unique R: two device buffers for pair chunks (and, unless S can be read in
// place, two for S chunks).  While chunk c is probed on the caller's stream,
// chunk c+1 is copied in on a copy stream and chunk c-1's pairs are copied
// out on another, so host<->device transfers overlap the lookups.  The host
// waits only for each chunk's pair count (8 bytes) before its copy-out.
// When S is page-locked host memory the GPU reads it in place (over
// NVLink-C2C on Grace-Blackwell, at a cost the latency-bound lookups hide) and
// no copy-in is issued.
// R with duplicates: per chunk, locate (first match and offsets per probe)
// -> expand the ranges into pairs -> copy out on alternating copy streams
// while the next chunk is located.
#include <algorithm>
#include <atomic>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace lj {
int probe_count_impl(const lj_index* idx, const uint64_t* S, uint64_t m, uint32_t* counts,
                     uint64_t* offsets, uint32_t* first, uint64_t* total_dev, uint64_t* total_host,
                     cudaStream_t s);
int probe_expand_impl(const uint32_t* first, const uint64_t* offsets, uint64_t m, lj_pair* pairs,
                      uint64_t cap, uint32_t s_base, cudaStream_t s);
int probe_emit_impl(const lj_index* idx, const uint64_t* S, uint64_t m, const uint64_t* offsets,
                    lj_pair* pairs, uint64_t cap, uint64_t* total_dev, uint64_t* total_host,
                    uint32_t s_base, cudaStream_t s);
}  // namespace lj

namespace {

struct Streams {
  cudaStream_t in = nullptr, out[2] = {nullptr, nullptr};
  cudaEvent_t ev[8] = {};
  ~Streams() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (in) cudaStreamDestroy(in);
    for (auto& o : out)
      if (o) cudaStreamDestroy(o);
  }
};

}  // namespace

namespace lj {
// probe keys per chunk of a host join (option "host_chunk")
std::atomic<uint64_t> g_host_chunk{1ull << 25};
void set_host_chunk(uint64_t v) { g_host_chunk = v; }
uint64_t get_host_chunk() { return g_host_chunk; }
}  // namespace lj

namespace {

}  // namespace

extern "C" int join_host(const lj_index* idx, const uint64_t* S_host, uint64_t m,
                         lj_pair* pairs_host, uint64_t capacity, uint64_t* written_host,
                         lj_stream_t stream) {
  using namespace lj;
  if (!idx) return fail(LJ_E_INVAL, "join_host: index is NULL");
  if (m >= (1ull << 32)) return fail(LJ_E_INVAL, "join_host: m must be below 2^32");
  if (m > 0 && !S_host) return fail(LJ_E_INVAL, "join_host: S is NULL");
  if (capacity > 0 && !pairs_host) return fail(LJ_E_INVAL, "join_host: pairs is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (m == 0) {
    if (written_host) *written_host = 0;
    return LJ_OK;
  }
  Streams st;
  LJ_CUDA(cudaStreamCreateWithFlags(&st.in, cudaStreamNonBlocking));
  LJ_CUDA(cudaStreamCreateWithFlags(&st.out[0], cudaStreamNonBlocking));
  LJ_CUDA(cudaStreamCreateWithFlags(&st.out[1], cudaStreamNonBlocking));
  for (auto& e : st.ev) LJ_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaEvent_t* in_done = st.ev;        // [2]
  cudaEvent_t* comp_done = st.ev + 2;  // [2]
  cudaEvent_t* out_done = st.ev + 4;   // [2]
  const uint64_t chunk = std::min<uint64_t>(m, std::max<uint64_t>(g_host_chunk.load(), 1u << 16));
  const uint64_t nchunks = (m + chunk - 1) / chunk;
  uint64_t written = 0;
  // page-locked (or registered) S can be read by the kernels in place
  const uint64_t* S_mapped = nullptr;
  {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, S_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer)
      S_mapped = (const uint64_t*)at.devicePointer;
    cudaGetLastError();   // clear a possible "not a CUDA pointer" error
  }

  if (idx->unique) {
    char* ws = nullptr;
    const size_t bytes = 4 * chunk * 8 + 256;
    LJ_CUDA(scratch_alloc((void**)&ws, bytes, s));
    uint64_t* Sd[2] = {(uint64_t*)ws, (uint64_t*)(ws + chunk * 8)};
    lj_pair* Pd[2] = {(lj_pair*)(ws + 2 * chunk * 8), (lj_pair*)(ws + 3 * chunk * 8)};
    uint64_t* tot_d = (uint64_t*)(ws + 4 * chunk * 8);
    // two page-locked counters per host thread, allocated on first use
    static thread_local uint64_t* tot_h = nullptr;
    if (!tot_h) LJ_CUDA(cudaMallocHost(&tot_h, 2 * sizeof(uint64_t)));
    int rc = 0;
    auto issue = [&](uint64_t c) -> int {
      const int b = (int)(c & 1);
      const uint64_t off = c * chunk, len = std::min(chunk, m - off);
      const uint64_t* Sc = Sd[b];
      if (S_mapped) {
        Sc = S_mapped + off;
      } else {
        // S buffer b was last read by compute(c-2)
        LJ_CUDA(cudaStreamWaitEvent(st.in, comp_done[b], 0));
        LJ_CUDA(cudaMemcpyAsync(Sd[b], S_host + off, len * 8, cudaMemcpyHostToDevice, st.in));
        LJ_CUDA(cudaEventRecord(in_done[b], st.in));
        LJ_CUDA(cudaStreamWaitEvent(s, in_done[b], 0));
      }
      LJ_CUDA(cudaStreamWaitEvent(s, out_done[b], 0));   // pair buffer b drained
      if (int r = probe_emit_impl(idx, Sc, len, nullptr, Pd[b], len, tot_d + b, nullptr,
                                  (uint32_t)off, s))
        return r;
      LJ_CUDA(cudaMemcpyAsync(tot_h + b, tot_d + b, 8, cudaMemcpyDeviceToHost, s));
      LJ_CUDA(cudaEventRecord(comp_done[b], s));
      return 0;
    };
    rc = issue(0);
    for (uint64_t c = 0; c < nchunks && !rc; ++c) {
      if (c + 1 < nchunks && (rc = issue(c + 1))) break;
      const int b = (int)(c & 1);
      if (cudaEventSynchronize(comp_done[b]) != cudaSuccess) {
        rc = fail(LJ_E_CUDA, "join_host: chunk %llu failed", (unsigned long long)c);
        break;
      }
      const uint64_t cnt = tot_h[b];
      const uint64_t room = capacity > written ? capacity - written : 0;
      const uint64_t take = std::min(cnt, room);
      // copy-outs alternate between two streams so consecutive ones overlap
      cudaStreamWaitEvent(st.out[b], comp_done[b], 0);
      if (take)
        cudaMemcpyAsync(pairs_host + written, Pd[b], take * 8, cudaMemcpyDeviceToHost, st.out[b]);
      cudaEventRecord(out_done[b], st.out[b]);
      written += cnt;
    }
    cudaStreamSynchronize(st.out[0]);
    cudaStreamSynchronize(st.out[1]);
    cudaStreamSynchronize(s);
    scratch_free(ws, s);
    cudaStreamSynchronize(s);
    if (rc) return rc;
  } else {
    // per chunk: locate (first match, offsets, |J| of the chunk) -> expand the
    // ranges into a pair buffer -> copy out on one of two copy streams while
    // the next chunk is located; a chunk waits for the copy-out of the chunk
    // two before it, so at most two pair buffers are in flight
    char* ws = nullptr;
    LJ_CUDA(scratch_alloc((void**)&ws, chunk * 8 + (chunk + 1) * 8 + chunk * 4 + 512, s));
    uint64_t* Sd = (uint64_t*)ws;
    uint64_t* off_d = (uint64_t*)(ws + chunk * 8);
    uint32_t* first_d = (uint32_t*)(ws + ((chunk * 16 + 8 + 255) & ~255ull));
    int rc = 0;
    for (uint64_t c = 0; c < nchunks && !rc; ++c) {
      const int b = (int)(c & 1);
      const uint64_t off = c * chunk, len = std::min(chunk, m - off);
      const uint64_t* Sc = Sd;
      if (S_mapped) {
        Sc = S_mapped + off;
      } else if (cudaMemcpyAsync(Sd, S_host + off, len * 8, cudaMemcpyHostToDevice, s) !=
                 cudaSuccess) {
        rc = fail(LJ_E_CUDA, "join_host: copy-in failed");
        break;
      }
      uint64_t cnt = 0;
      if ((rc = probe_count_impl(idx, Sc, len, nullptr, off_d, first_d, nullptr, &cnt, s))) break;
      const uint64_t room = capacity > written ? capacity - written : 0;
      const uint64_t take = std::min(cnt, room);
      if (take) {
        if (cudaStreamWaitEvent(s, out_done[b], 0) != cudaSuccess) {   // chunk c-2 copied out
          rc = fail(LJ_E_CUDA, "join_host: stream wait failed");
          break;
        }
        lj_pair* Pd = nullptr;
        if (scratch_alloc((void**)&Pd, take * 8, s) != cudaSuccess) {
          rc = fail(LJ_E_NOMEM, "join_host: no room for %llu pairs", (unsigned long long)take);
          break;
        }
        if ((rc = probe_expand_impl(first_d, off_d, len, Pd, take, (uint32_t)off, s))) break;
        cudaEventRecord(comp_done[b], s);
        cudaStreamWaitEvent(st.out[b], comp_done[b], 0);
        cudaMemcpyAsync(pairs_host + written, Pd, take * 8, cudaMemcpyDeviceToHost, st.out[b]);
        scratch_free(Pd, st.out[b]);
        cudaEventRecord(out_done[b], st.out[b]);
      }
      written += cnt;
    }
    cudaStreamSynchronize(st.out[0]);
    cudaStreamSynchronize(st.out[1]);
    cudaStreamSynchronize(s);
    scratch_free(ws, s);
    cudaStreamSynchronize(s);
    if (rc) return rc;
  }
  if (written_host) *written_host = written;
  // a capacity overflow inside a chunk (take < cnt) also sets the device word
  const int dev_rc = take_device_errors(idx->device, s);
  if (written > capacity)
    return fail(LJ_E_CAPACITY, "join_host: %llu pairs do not fit the capacity of %llu",
                (unsigned long long)written, (unsigned long long)capacity);
  return dev_rc;
}
