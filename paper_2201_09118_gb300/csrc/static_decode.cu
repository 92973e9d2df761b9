// static_decode.cu -- hd_decode_static: gap-array decode that allocates no
// memory.  Its scratch (control words, look-back states, decode table) lives
// in a fixed file-scope device array instead of a context's cudaMalloc'd
// workspace.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "hd.h"
#include "kernels.h"

namespace {

// Scratch shared by every hd_decode_static call on a device (1 MiB).
constexpr size_t kStaticScratchBytes = static_cast<size_t>(1) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};  // device address per device
int g_num_sms[kMaxDevices] = {};

constexpr uint32_t kThreads = 256;
constexpr uint32_t kWindow = 4096;
constexpr uint32_t kLutBits = 12;
constexpr uint64_t kTimeoutCycles = 4000000000ull;  // ~2 s at GB300 clocks

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Scratch symbols per thread: about 1.5x the expected codewords of a
// subsequence, a multiple of 8, at most S.
uint32_t scratch_syms(uint32_t S, uint64_t nbits, uint64_t n) {
  const double per = static_cast<double>(S) * static_cast<double>(n) / static_cast<double>(nbits);
  uint32_t c = static_cast<uint32_t>(per * 1.35 + 4.0);
  c = (c + 7) / 8 * 8;
  return c > S ? S : c;
}

// One-time set-up on the current device: the device address of the scratch
// array (host code may not use the symbol itself) and the SM count.
int setup_device(int dev, unsigned char** ptr, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    g_num_sms[dev] = n;
  }
  *ptr = g_scratch_ptr[dev];
  *sms = g_num_sms[dev];
  return HD_OK;
}

}  // namespace

extern "C" int hd_decode_static(const hd_field* f, uint16_t* d_out, void* stream) {
  if (!f || !f->gap || !f->lengths || !f->words) return HD_ERR_ARG;
  if (f->subseq_bits != 64 && f->subseq_bits != 128 && f->subseq_bits != 256) return HD_ERR_ARG;
  if (f->alphabet < 2 || f->alphabet > 65536) return HD_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(f->words) & 15u) return HD_ERR_ARG;
  if (f->nwords * 32 < f->nbits) return HD_ERR_ARG;
  if (f->n == 0 && f->nbits == 0) return HD_OK;
  if (f->n == 0 || f->nbits == 0) return HD_ERR_CORRUPT;
  if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 1u)) return HD_ERR_ARG;

  hd::LaunchShape s{};
  s.S = f->subseq_bits;
  s.threads = kThreads;
  s.window = kWindow;
  s.K = kLutBits;
  s.cmax = scratch_syms(s.S, f->nbits, f->n);
  s.long_cap = ((f->alphabet < 4096 ? f->alphabet : 4096u) + 7u) / 8 * 8;
  s.grid = 0;
  const uint64_t nsub = (f->nbits + s.S - 1) / s.S;
  const uint64_t units = (nsub + s.threads - 1) / s.threads;  // tiles

  // scratch layout: ticket, abort flag, error word | tile states | table
  const size_t err_off = 8;
  const size_t state_off = 16;
  const size_t zero_bytes = round_up(state_off + 8 * units, 16);
  const size_t tab_off = round_up(zero_bytes, 256);
  const size_t need = tab_off + hd::table_bytes(s.K, f->alphabet);
  if (units > (kStaticScratchBytes / 8) || need > kStaticScratchBytes) return HD_ERR_CAPACITY;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  unsigned char* scratch = nullptr;
  int num_sms = 0;
  int rc = setup_device(dev, &scratch, &num_sms);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  hd::FieldDesc d;
  std::memset(&d, 0, sizeof(d));
  d.words = f->words;
  d.nwords = f->nwords;
  d.nbits = f->nbits;
  d.nsub = nsub;
  d.gap = f->gap;
  d.gap_stride = 1;
  d.alphabet = f->alphabet;
  d.lengths = f->lengths;
  d.table = reinterpret_cast<const hd::TableHeader*>(scratch + tab_off);
  d.out = d_out;
  d.n = f->n;
  d.unit_begin = 0;
  d.nunits = units;
  d.err = reinterpret_cast<uint32_t*>(scratch + err_off);

  hd::PrepParams pp{};
  pp.f0 = d;
  pp.fields = nullptr;
  pp.nfields = 1;
  pp.table_blocks = 1;
  pp.K = s.K;
  pp.zero_ptr = reinterpret_cast<uint4*>(scratch);
  pp.zero_vec = zero_bytes / 16;
  pp.zero_blocks = 1;
  if (hd::launch_prepare(pp, st) != cudaSuccess) return HD_ERR_CUDA;

  hd::DecodeParams dp{};
  dp.f0 = d;
  dp.fields = nullptr;
  dp.nfields = 1;
  dp.K = s.K;
  dp.window = s.window;
  dp.cmax = s.cmax;
  dp.long_cap = s.long_cap;
  dp.total_units = units;
  dp.unit_state = reinterpret_cast<uint64_t*>(scratch + state_off);
  dp.ticket = reinterpret_cast<uint32_t*>(scratch);
  dp.abort_flag = reinterpret_cast<uint32_t*>(scratch) + 1;
  dp.timeout_cycles = kTimeoutCycles;
  if (hd::launch_decode_single_pass(dp, s, num_sms, st) != cudaSuccess) return HD_ERR_CUDA;

  uint32_t bits = 0;
  if (cudaMemcpyAsync(&bits, scratch + err_off, sizeof(bits), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  if (!bits) return HD_OK;
  if (bits & hd::kErrTimeout) return HD_ERR_TIMEOUT;
  if (bits & hd::kErrTable) return HD_ERR_ARG;
  return HD_ERR_CORRUPT;
}
