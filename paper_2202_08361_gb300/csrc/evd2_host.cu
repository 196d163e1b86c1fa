// evd2_host.cu -- jsvd_evd2x2_batched_host: the batched 2x2 EVD on host
// buffers.
//
// Two ways to move the data, the same kernel and bits either way:
//
// Direct (default, when every stream is page-locked memory mapped for the
// current device): the EVD kernel reads its inputs from the host streams
// and writes its outputs back to them over the host link; no staging copy,
// one launch.  On a coherent CPU-GPU node the link then carries exactly the
// streams' bytes, both directions at once.
//
// Staged (pageable or unmapped buffers, or JSVD_TUNE_EVD_HOST = 1): the
// batch is cut into chunks.  Chunk c uses workspace slot c mod kSlots and
// internal stream c mod kSlots: the copies of its input streams to the
// slot, the EVD kernel on the slot, the copies of its output streams back.
// With three slots the host-to-device copy of one chunk, the kernel of the
// next older one and the device-to-host copy of the oldest run at the same
// time (the two copy directions use separate copy engines).  Events order
// the internal streams after the work already queued on the caller's
// stream, and the caller's stream after all chunks, so the call behaves
// like one asynchronous operation on `stream`.
#include <mutex>

#include "common.cuh"
#include "jsvd_internal.h"

namespace jsvd {

constexpr int kSlots = 3;
static int g_host_path = 0;  // 0: direct when every stream is mapped; 1: always staged
constexpr int64_t kChunk = int64_t(1) << 20;  // matrices per chunk

// bytes of one slot: 4 input and 5 output double streams, one int32 stream
static size_t slot_bytes(int64_t chunk) { return (size_t)chunk * (9 * sizeof(double) + 4); }

struct HostPipe {
  bool init = false;
  cudaStream_t st[kSlots];
};

static std::mutex g_pipe_mu;
static HostPipe g_pipe[64];  // per device ordinal

static int pipe_streams(cudaStream_t *out)
{
  int dev = 0;
  JSVD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return JSVD_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe &p = g_pipe[dev];
  if (!p.init) {
    for (int k = 0; k < kSlots; ++k)
      JSVD_CUDA(cudaStreamCreateWithFlags(&p.st[k], cudaStreamNonBlocking));
    p.init = true;
  }
  for (int k = 0; k < kSlots; ++k) out[k] = p.st[k];
  return JSVD_OK;
}

// Events of one call, destroyed on every return path (destroying a
// recorded event is allowed: its resources go once it has fired).
struct CallEvents {
  cudaEvent_t ev[kSlots + 1] = {};
  int made = 0;
  int create()
  {
    for (; made < kSlots + 1; ++made)
      JSVD_CUDA(cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming));
    return JSVD_OK;
  }
  ~CallEvents()
  {
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  }
};

static int copy_in(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
  if (src) JSVD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
  return JSVD_OK;
}

static int copy_out(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
  if (dst) JSVD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st));
  return JSVD_OK;
}

// The address through which the current device reads and writes the host
// range [p, p + bytes), or nullptr when the range is not page-locked memory
// mapped for it.  Both ends are checked (a stream is one buffer).
static void *mapped_address(const void *p, size_t bytes)
{
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a0, a1;
  const char *last = static_cast<const char *>(p) + (bytes - 1);
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();  // an unregistered pointer is an answer here, not an error
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost) return nullptr;
  if (!a0.devicePointer || !a1.devicePointer) return nullptr;
  // one linear mapping across the range
  if ((char *)a1.devicePointer - (char *)a0.devicePointer != (ptrdiff_t)(bytes - 1)) return nullptr;
  return a0.devicePointer;
}

// Device addresses of all given host streams in *d, true when every one is
// mapped.
static bool map_streams(const jsvd_evd2_streams *h, int64_t n, bool cplx, jsvd_evd2_streams *d)
{
  const size_t b = (size_t)n * sizeof(double);
  bool ok = true;
  auto in = [&](const double *x) -> const double * {
    if (!x) return nullptr;
    void *m = mapped_address(x, b);
    ok = ok && m;
    return static_cast<const double *>(m);
  };
  auto out = [&](double *x) -> double * {
    if (!x) return nullptr;
    void *m = mapped_address(x, b);
    ok = ok && m;
    return static_cast<double *>(m);
  };
  d->a11 = in(h->a11);
  d->a22 = in(h->a22);
  d->a21_re = in(h->a21_re);
  d->a21_im = cplx ? in(h->a21_im) : nullptr;
  d->cos_phi = out(h->cos_phi);
  d->ea_tan_re = out(h->ea_tan_re);
  d->ea_tan_im = cplx ? out(h->ea_tan_im) : nullptr;
  d->lambda1 = out(h->lambda1);
  d->lambda2 = out(h->lambda2);
  d->zeta_p = nullptr;
  if (h->zeta_p) {
    void *m = mapped_address(h->zeta_p, (size_t)n * sizeof(int32_t));
    ok = ok && m;
    d->zeta_p = static_cast<int32_t *>(m);
  }
  return ok;
}

int evd2_set_host_path(int v)
{
  if (v < 0 || v > 1) return -2;
  g_host_path = v;
  return JSVD_OK;
}

}  // namespace jsvd

using namespace jsvd;

extern "C" int jsvd_evd2x2_host_workspace_size(size_t *bytes)
{
  if (!bytes) return -1;
  *bytes = kSlots * slot_bytes(kChunk);
  return JSVD_OK;
}

extern "C" int jsvd_evd2x2_batched_host(jsvd_field field, const jsvd_evd2_streams *h, int64_t n,
                                        void *work, size_t work_bytes, void *stream)
{
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  if (!h) return -2;
  if (n < 0) return -3;
  if (n == 0) return JSVD_OK;
  const bool cplx = (field == JSVD_COMPLEX);
  if (!h->a11 || !h->a22 || !h->a21_re || !h->cos_phi || !h->ea_tan_re) return -2;
  if (cplx && (!h->a21_im || !h->ea_tan_im)) return -2;
  if (!work || ((uintptr_t)work & 255)) return -4;
  if (work_bytes < kSlots * slot_bytes(kChunk)) return JSVD_E_WORKSPACE;
  if (g_host_path == 0) {
    jsvd_evd2_streams d;
    if (map_streams(h, n, cplx, &d)) return jsvd_evd2x2_batched(field, &d, n, stream);
  }
  cudaStream_t ps[kSlots];
  JSVD_TRY(pipe_streams(ps));
  cudaStream_t user = as_stream(stream);
  CallEvents E;
  JSVD_TRY(E.create());
  cudaEvent_t start = E.ev[0], *done = E.ev + 1;
  JSVD_CUDA(cudaEventRecord(start, user));
  for (int k = 0; k < kSlots; ++k) JSVD_CUDA(cudaStreamWaitEvent(ps[k], start, 0));
  const size_t D = sizeof(double);
  for (int64_t c0 = 0, c = 0; c0 < n; c0 += kChunk, ++c) {
    const int k = (int)(c % kSlots);
    const int64_t len = (n - c0 < kChunk) ? (n - c0) : kChunk;
    double *slot = reinterpret_cast<double *>((char *)work + (size_t)k * slot_bytes(kChunk));
    jsvd_evd2_streams d;
    d.a11 = slot;
    d.a22 = slot + kChunk;
    d.a21_re = slot + 2 * kChunk;
    d.a21_im = cplx ? slot + 3 * kChunk : nullptr;
    d.cos_phi = slot + 4 * kChunk;
    d.ea_tan_re = slot + 5 * kChunk;
    d.ea_tan_im = cplx ? slot + 6 * kChunk : nullptr;
    d.lambda1 = h->lambda1 ? slot + 7 * kChunk : nullptr;
    d.lambda2 = h->lambda2 ? slot + 8 * kChunk : nullptr;
    d.zeta_p = h->zeta_p ? reinterpret_cast<int32_t *>(slot + 9 * kChunk) : nullptr;
    cudaStream_t st = ps[k];
    const size_t b = (size_t)len * D;
    JSVD_TRY(copy_in((void *)d.a11, h->a11 + c0, b, st));
    JSVD_TRY(copy_in((void *)d.a22, h->a22 + c0, b, st));
    JSVD_TRY(copy_in((void *)d.a21_re, h->a21_re + c0, b, st));
    if (cplx) JSVD_TRY(copy_in((void *)d.a21_im, h->a21_im + c0, b, st));
    const int rc = jsvd_evd2x2_batched(field, &d, len, st);
    if (rc) return rc;
    JSVD_TRY(copy_out(h->cos_phi + c0, d.cos_phi, b, st));
    JSVD_TRY(copy_out(h->ea_tan_re + c0, d.ea_tan_re, b, st));
    if (cplx) JSVD_TRY(copy_out(h->ea_tan_im + c0, d.ea_tan_im, b, st));
    if (h->lambda1) JSVD_TRY(copy_out(h->lambda1 + c0, d.lambda1, b, st));
    if (h->lambda2) JSVD_TRY(copy_out(h->lambda2 + c0, d.lambda2, b, st));
    if (h->zeta_p) JSVD_TRY(copy_out(h->zeta_p + c0, d.zeta_p, (size_t)len * 4, st));
  }
  for (int k = 0; k < kSlots; ++k) {
    JSVD_CUDA(cudaEventRecord(done[k], ps[k]));
    JSVD_CUDA(cudaStreamWaitEvent(user, done[k], 0));
  }
  return JSVD_OK;
}
