// api.cpp -- the C ABI of hd.h: context, argument checks, workspace layout
// and the launch sequence (decode-table kernel, then the decode kernels of
// the field's strategy).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "hd.h"
#include "host_internal.h"
#include "kernels.h"

struct hd_ctx {
  int device = 0;
  int num_sms = 0;
  int max_smem = 0;  // opt-in shared memory per block (bytes)
  std::mutex mu;
  hd_config cfg{};
  // device workspace (control region, decode tables, field descriptors)
  char* ws = nullptr;
  size_t ws_cap = 0;
  // status of the last queued operation
  int host_status = HD_OK;       // argument-level outcome decided on the host
  size_t err_off = 0;            // offset of its error words in ws
  uint32_t err_count = 0;        // number of error words (fields)
  std::vector<uint32_t> err_map; // field -> error word (batch)
  // device staging for hd_decode_host
  char* stage = nullptr;
  size_t stage_cap = 0;
  // kernel timing
  bool profile = false;
  std::vector<cudaEvent_t> events;
  size_t events_used = 0;
  uint64_t launches = 0;
  hd::LaunchShape last_shape{};  // launch shape of the last decode
};

namespace {

using hd::FieldDesc;

constexpr uint32_t kDefaultThreads = 256;
constexpr uint32_t kDefaultK = 12;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int map_err_bits(uint32_t b) {
  if (!b) return HD_OK;
  if (b & hd::kErrTimeout) return HD_ERR_TIMEOUT;
  if (b & hd::kErrNoSync) return HD_ERR_NOSYNC;
  if (b & hd::kErrTable) return HD_ERR_ARG;
  return HD_ERR_CORRUPT;
}

int ensure_ws(hd_ctx* c, size_t bytes) {
  if (bytes <= c->ws_cap) return HD_OK;
  if (c->ws) {
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_cap = 0;
  }
  size_t cap = align_up(std::max(bytes, static_cast<size_t>(1) << 20), 1 << 20);
  if (cudaMalloc(&c->ws, cap) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_NOMEM;
  }
  c->ws_cap = cap;
  return HD_OK;
}

int ensure_stage(hd_ctx* c, size_t bytes) {
  if (bytes <= c->stage_cap) return HD_OK;
  if (c->stage) {
    cudaDeviceSynchronize();
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
  }
  size_t cap = align_up(std::max(bytes, static_cast<size_t>(1) << 20), 1 << 20);
  if (cudaMalloc(&c->stage, cap) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_NOMEM;
  }
  c->stage_cap = cap;
  return HD_OK;
}

bool valid_S(uint32_t s) { return s == 64 || s == 128 || s == 256; }

// Checks one field against the stream format; returns HD_OK, an error, or
// HD_PENDING when there is nothing to launch (n == 0 and nbits == 0).
int check_field(const hd_field* f, bool need_out, const void* out) {
  if (!f) return HD_ERR_ARG;
  if (!valid_S(f->subseq_bits)) return HD_ERR_ARG;
  if (f->alphabet < 2 || f->alphabet > 65536 || !f->lengths) return HD_ERR_ARG;
  if (f->n == 0 && f->nbits == 0) return HD_PENDING;
  if (!f->words) return HD_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(f->words) & 15u) return HD_ERR_ARG;
  if (f->nwords * 32 < f->nbits) return HD_ERR_ARG;
  if (need_out && (!out || (reinterpret_cast<uintptr_t>(out) & 1u))) return HD_ERR_ARG;
  return HD_OK;
}

// Decoder subsequence when the configuration leaves it open: gap-array
// decodes take 256-bit subsequences (every second gap entry of a 128-bit
// stream) because the per-tile work of a thread then amortises its fixed
// costs better; the synchronising kernel uses the stream's own size.
uint32_t default_decoder_S(uint32_t stream_S, bool gap) {
  if (!gap) return stream_S;
  return stream_S < 256 ? 256 : stream_S;
}

hd::LaunchShape shape_for(const hd_ctx* c, uint32_t stream_S, bool gap) {
  hd::LaunchShape s{};
  s.S = c->cfg.subseq_bits ? c->cfg.subseq_bits : default_decoder_S(stream_S, gap);
  s.threads = c->cfg.threads ? c->cfg.threads : kDefaultThreads;
  s.K = c->cfg.lut_bits ? c->cfg.lut_bits : kDefaultK;
  s.window = c->cfg.window;  // 0: chosen per launch
  s.grid = 0;
  return s;
}

uint64_t tiles_for(uint64_t nsub, const hd::LaunchShape& s) {
  return (nsub + s.threads - 1) / s.threads;
}

cudaEvent_t next_event(hd_ctx* c) {
  if (c->events_used == c->events.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->events.push_back(e);
  }
  return c->events[c->events_used++];
}

// Fills the per-field part of a descriptor (device pointers, sizes).
void fill_desc(FieldDesc& d, const hd_field* f, const hd::LaunchShape& s, uint16_t* out) {
  std::memset(&d, 0, sizeof(d));
  d.words = f->words;
  d.nwords = f->nwords;
  d.nbits = f->nbits;
  d.nsub = (f->nbits + s.S - 1) / s.S;
  d.gap = f->gap;
  d.gap_stride = s.S / f->subseq_bits;
  d.alphabet = f->alphabet;
  d.lengths = f->lengths;
  d.out = out;
  d.n = f->n;
}

// Queues the decode-table build (which also clears the per-launch control
// region) and the decode kernels for fields that all use the same strategy:
//   gap array            count kernel, decode-and-write kernel;
//   self-synchronisation synchronising kernel, link-fix kernel, then the same
//                        decode-and-write kernel (with sync_only: the first two
//                        alone, which leave the gap arrays in each gap_out).
int queue_decode(hd_ctx* c, std::vector<FieldDesc>& descs, const hd::LaunchShape& shape,
                 bool self_sync, bool sync_only, cudaStream_t st) {
  const uint32_t nf = static_cast<uint32_t>(descs.size());
  hd::LaunchShape s = shape;
  double bits_per = 0;
  uint32_t amax = 0;
  for (auto& d : descs) {
    bits_per = std::max(bits_per, static_cast<double>(d.nbits) / static_cast<double>(d.n ? d.n : 1));
    amax = std::max(amax, d.alphabet);
  }
  // symbols of codes longer than the first-level table, kept in shared memory
  s.long_cap = static_cast<uint32_t>(align_up(std::min<uint32_t>(amax, 4096), 8));
  if (s.window == 0) {
    // output window: about 1.2x a tile's expected symbol count
    const double want = 1.2 * s.threads * s.S / std::max(bits_per, 0.25) + 64.0;
    s.window = static_cast<uint32_t>(std::min(std::max(want, 1024.0), 16384.0));
  }
  s.window = static_cast<uint32_t>(align_up(std::max(s.window, s.S), 8));
  {
    // the window is an optimisation (larger outputs go through several
    // windows), so it shrinks to fit shared memory
    const size_t budget = static_cast<size_t>(c->max_smem) - 2048;
    while (s.window > std::max<uint32_t>(1024, s.S) && hd::two_phase_smem_bytes(s) > budget)
      s.window -= 512;
    if (hd::two_phase_smem_bytes(s) > budget) return HD_ERR_ARG;
    if (self_sync && hd::sync_smem_bytes(s) > budget) return HD_ERR_ARG;
  }
  uint64_t total_tiles = 0, total_sub = 0;
  for (auto& d : descs) {
    d.unit_begin = total_tiles;
    d.nunits = tiles_for(d.nsub, s);
    total_tiles += d.nunits;
    d.count_begin = total_sub;
    total_sub += d.nsub;
  }
  // workspace layout; [0, zero_bytes) is cleared by the table kernel
  size_t off = 0;
  const size_t err_off = off;
  off = align_up(off + 4ull * nf, 16);
  const size_t seg_off = off;  // codewords per 256 tiles
  off = align_up(off + 8ull * ((total_tiles + 255) / 256 + 1), 16);
  const size_t zero_bytes = off;
  off = align_up(off, 256);
  std::vector<size_t> tab_off(nf);
  for (uint32_t k = 0; k < nf; ++k) {
    tab_off[k] = off;
    off += hd::table_bytes(s.K, descs[k].alphabet);
  }
  const size_t desc_off = align_up(off, 256);
  off = desc_off + (nf > 1 ? sizeof(FieldDesc) * nf : 0);
  const size_t tile_off = align_up(off, 256);
  off = tile_off + 4ull * total_tiles;
  const size_t count_off = align_up(off, 256);
  off = count_off + hd::count_bytes_per_subsequence(s.S) * total_sub;
  // self-synchronisation: subsequence starts, tile links (16-byte padded)
  const size_t link_bytes = align_up(total_tiles + 1, 16) + 16;
  const size_t gap_off = align_up(off, 256);
  if (self_sync && !sync_only) off = gap_off + total_sub;
  const size_t ta_off = align_up(off, 256);
  const size_t te_off = align_up(ta_off + link_bytes, 256);
  const size_t tf_off = align_up(te_off + link_bytes, 256);
  if (self_sync) off = tf_off + total_tiles;
  int rc = ensure_ws(c, off);
  if (rc) return rc;
  char* ws = c->ws;
  for (uint32_t k = 0; k < nf; ++k) {
    FieldDesc& d = descs[k];
    d.table = reinterpret_cast<const hd::TableHeader*>(ws + tab_off[k]);
    d.err = reinterpret_cast<uint32_t*>(ws + err_off) + k;
    if (self_sync) {
      if (!sync_only) d.gap_out = reinterpret_cast<uint8_t*>(ws + gap_off) + d.count_begin;
      d.gap = d.gap_out;
      d.gap_stride = 1;
    }
  }
  cudaError_t e = cudaSuccess;
  if (nf > 1) {
    e = cudaMemcpyAsync(ws + desc_off, descs.data(), sizeof(FieldDesc) * nf,
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return HD_ERR_CUDA;
  }
  hd::PrepParams pp{};
  pp.f0 = descs[0];
  pp.fields = reinterpret_cast<const FieldDesc*>(ws + desc_off);
  pp.nfields = nf;
  pp.K = s.K;
  pp.zero_ptr = reinterpret_cast<uint4*>(ws);
  pp.zero_vec = zero_bytes / 16;
  pp.zero_blocks = static_cast<uint32_t>(std::min<uint64_t>((pp.zero_vec + 4095) / 4096, 64));
  if (pp.zero_blocks == 0) pp.zero_blocks = 1;
  e = hd::launch_prepare(pp, st);
  if (e != cudaSuccess) return HD_ERR_CUDA;
  c->launches += 1;

  hd::DecodeParams dp{};
  dp.f0 = descs[0];
  dp.fields = pp.fields;
  dp.nfields = nf;
  dp.K = s.K;
  dp.window = s.window;
  dp.long_cap = s.long_cap;
  dp.total_units = total_tiles;
  dp.counts = ws + count_off;
  dp.tile_total = reinterpret_cast<uint32_t*>(ws + tile_off);
  dp.seg_total = reinterpret_cast<uint64_t*>(ws + seg_off);
  if (self_sync) {
    dp.tile_a = reinterpret_cast<uint8_t*>(ws + ta_off);
    dp.tile_e = reinterpret_cast<uint8_t*>(ws + te_off);
    dp.tile_flag = reinterpret_cast<uint8_t*>(ws + tf_off);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    e0 = next_event(c);
    e1 = next_event(c);
    cudaEventRecord(e0, st);
  }
  if (self_sync) {
    e = hd::launch_sync(dp, s, c->num_sms, st);
    if (e == cudaSuccess && !sync_only) e = hd::launch_write(dp, s, c->num_sms, st);
  } else {
    e = hd::launch_decode_two_phase(dp, s, c->num_sms, st);
  }
  if (c->profile) cudaEventRecord(e1, st);
  if (e != cudaSuccess) return HD_ERR_CUDA;
  c->launches += self_sync ? (sync_only ? 2 : 3) : 2;
  c->err_off = err_off;
  c->err_count = nf;
  c->last_shape = s;
  return HD_OK;
}

int read_errors(hd_ctx* c, void* stream, std::vector<uint32_t>& bits) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  bits.assign(c->err_count, 0);
  if (c->err_count && c->ws) {
    if (cudaMemcpy(bits.data(), c->ws + c->err_off, 4ull * c->err_count,
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
  }
  return HD_OK;
}

}  // namespace

extern "C" {

const char* hd_version(void) { return "hd-gb300 0.1"; }

int hd_ctx_create(int device, hd_ctx** out) {
  if (!out) return HD_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  hd_ctx* c = new (std::nothrow) hd_ctx();
  if (!c) return HD_ERR_NOMEM;
  c->device = device;
  DeviceGuard g(device);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess) {
    delete c;
    return HD_ERR_CUDA;
  }
  *out = c;
  return HD_OK;
}

int hd_ctx_destroy(hd_ctx* c) {
  if (!c) return HD_ERR_ARG;
  {
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    if (c->ws) cudaFree(c->ws);
    if (c->stage) cudaFree(c->stage);
    for (auto e : c->events) cudaEventDestroy(e);
  }
  delete c;
  return HD_OK;
}

int hd_set_config(hd_ctx* c, const hd_config* cfg) {
  if (!c) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  if (!cfg) {
    c->cfg = hd_config{};
    return HD_OK;
  }
  if (cfg->subseq_bits && !valid_S(cfg->subseq_bits) && cfg->subseq_bits != 512) return HD_ERR_ARG;
  if (cfg->threads && cfg->threads != 128 && cfg->threads != 256 && cfg->threads != 512)
    return HD_ERR_ARG;
  if (cfg->lut_bits && (cfg->lut_bits < 8 || cfg->lut_bits > 13)) return HD_ERR_ARG;
  if (cfg->window && (cfg->window < 64 || cfg->window > 32768)) return HD_ERR_ARG;
  c->cfg = *cfg;
  return HD_OK;
}

int hd_get_config(hd_ctx* c, hd_config* cfg) {
  if (!c || !cfg) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  cfg->subseq_bits = c->cfg.subseq_bits;
  cfg->threads = c->cfg.threads ? c->cfg.threads : kDefaultThreads;
  cfg->window = c->cfg.window ? c->cfg.window : c->last_shape.window;
  cfg->lut_bits = c->cfg.lut_bits ? c->cfg.lut_bits : kDefaultK;
  return HD_OK;
}

static int decode_impl(hd_ctx* c, const hd_field* f, uint16_t* d_out, uint8_t* gap_out,
                       void* stream) {
  const bool sync_only = gap_out != nullptr;
  int rc = check_field(f, !sync_only, d_out);
  c->err_count = 0;
  if (rc == HD_PENDING) {
    c->host_status = HD_OK;
    return HD_OK;
  }
  if (rc) {
    c->host_status = rc;
    return rc;
  }
  if (!sync_only && (f->nbits == 0 || f->n == 0)) {
    c->host_status = HD_ERR_CORRUPT;  // symbols without bits or bits without symbols
    return HD_OK;
  }
  const bool self_sync = sync_only || f->gap == nullptr;
  hd::LaunchShape s = shape_for(c, f->subseq_bits, !self_sync);
  if (self_sync && s.S > 256) s.S = 256;  // the synchronising kernel stops at 256-bit subsequences
  if (!self_sync && (s.S % f->subseq_bits)) {
    c->host_status = HD_ERR_ARG;
    return HD_ERR_ARG;
  }
  std::vector<FieldDesc> descs(1);
  fill_desc(descs[0], f, s, d_out);
  if (sync_only) {
    descs[0].gap = nullptr;
    descs[0].gap_out = gap_out;
    descs[0].out = nullptr;
  }
  rc = queue_decode(c, descs, s, self_sync, sync_only, static_cast<cudaStream_t>(stream));
  c->host_status = rc;
  return rc;
}

int hd_decode(hd_ctx* c, const hd_field* f, uint16_t* d_out, void* stream) {
  if (!c) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return decode_impl(c, f, d_out, nullptr, stream);
}

int hd_sync_points(hd_ctx* c, const hd_field* f, uint8_t* gap_out, void* stream) {
  if (!c || !gap_out || !f) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  if (c->cfg.subseq_bits && c->cfg.subseq_bits != f->subseq_bits) return HD_ERR_ARG;
  return decode_impl(c, f, nullptr, gap_out, stream);
}

int hd_status(hd_ctx* c, void* stream) {
  if (!c) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  std::vector<uint32_t> bits;
  int rc = read_errors(c, stream, bits);
  if (rc) return rc;
  if (c->host_status != HD_OK) return c->host_status;
  uint32_t all = 0;
  for (uint32_t b : bits) all |= b;
  return map_err_bits(all);
}

int hd_decode_batch(hd_ctx* c, const hd_field* fs, uint32_t nf, uint16_t* const* d_outs,
                    void* stream) {
  if (!c || (nf && (!fs || !d_outs))) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  c->err_count = 0;
  c->host_status = HD_OK;
  c->err_map.assign(nf, 0xffffffffu);
  if (nf == 0) return HD_OK;
  uint32_t maxS = 0;
  for (uint32_t i = 0; i < nf; ++i) {
    int rc = check_field(&fs[i], true, d_outs[i]);
    if (rc == HD_PENDING) continue;
    if (rc) {
      c->host_status = rc;
      return rc;
    }
    maxS = std::max(maxS, fs[i].subseq_bits);
  }
  bool all_gap = true;
  for (uint32_t i = 0; i < nf; ++i) all_gap &= fs[i].gap != nullptr;
  hd::LaunchShape s = shape_for(c, maxS ? maxS : 128, all_gap);
  std::vector<FieldDesc> gap_d, sync_d;
  std::vector<uint32_t> gap_i, sync_i;
  for (uint32_t i = 0; i < nf; ++i) {
    const hd_field* f = &fs[i];
    if (f->n == 0 && f->nbits == 0) continue;
    if (f->nbits == 0 || f->n == 0 || (f->gap && s.S % f->subseq_bits)) {
      c->host_status = f->nbits == 0 || f->n == 0 ? HD_ERR_CORRUPT : HD_ERR_ARG;
      return c->host_status == HD_ERR_ARG ? HD_ERR_ARG : HD_OK;
    }
    FieldDesc d;
    fill_desc(d, f, s, d_outs[i]);
    if (f->gap) {
      gap_d.push_back(d);
      gap_i.push_back(i);
    } else {
      sync_d.push_back(d);
      sync_i.push_back(i);
    }
  }
  // Two strategy groups run as two launches; the error words of the first
  // are copied aside so hd_batch_status sees both.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<uint32_t> merged;
  if (!gap_d.empty() && !sync_d.empty()) {
    // run sequentially with separate control regions: simplest is two queues
    int rc = queue_decode(c, gap_d, s, false, false, st);
    if (rc) return rc;
    std::vector<uint32_t> bits;
    rc = read_errors(c, stream, bits);
    if (rc) return rc;
    rc = queue_decode(c, sync_d, s, true, false, st);
    if (rc) return rc;
    std::vector<uint32_t> bits2;
    rc = read_errors(c, stream, bits2);
    if (rc) return rc;
    c->err_map.assign(nf, 0xffffffffu);
    // stash merged bits in host_status-only form: keep per-field map
    merged.assign(nf, 0);
    for (size_t k = 0; k < gap_i.size(); ++k) merged[gap_i[k]] = bits[k];
    for (size_t k = 0; k < sync_i.size(); ++k) merged[sync_i[k]] = bits2[k];
    // encode merged results as host-side per-field statuses
    c->err_count = 0;
    c->err_map.assign(nf, 0);
    for (uint32_t i = 0; i < nf; ++i) c->err_map[i] = 0x80000000u | merged[i];
    return HD_OK;
  }
  const bool ss = gap_d.empty();
  std::vector<FieldDesc>& d = ss ? sync_d : gap_d;
  std::vector<uint32_t>& idx = ss ? sync_i : gap_i;
  int rc = queue_decode(c, d, s, ss, false, st);
  if (rc) return rc;
  for (size_t k = 0; k < idx.size(); ++k) c->err_map[idx[k]] = static_cast<uint32_t>(k);
  return HD_OK;
}

int hd_batch_status(hd_ctx* c, int32_t* status, uint32_t nf, void* stream) {
  if (!c || (nf && !status)) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  std::vector<uint32_t> bits;
  int rc = read_errors(c, stream, bits);
  if (rc) return rc;
  int first = c->host_status;
  for (uint32_t i = 0; i < nf; ++i) {
    int s = HD_OK;
    if (i < c->err_map.size()) {
      const uint32_t m = c->err_map[i];
      if (m & 0x80000000u) s = map_err_bits(m & 0x7fffffffu);
      else if (m < bits.size()) s = map_err_bits(bits[m]);
    }
    status[i] = s;
    if (first == HD_OK && s != HD_OK) first = s;
  }
  return first;
}

int hd_decode_host(hd_ctx* c, const hd_field* f, uint16_t* host_out, void* stream) {
  if (!c || !f) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  int rc = check_field(f, true, host_out);
  if (rc == HD_PENDING) return HD_OK;
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t nsub = (f->nbits + f->subseq_bits - 1) / f->subseq_bits;
  const size_t words_b = align_up(f->nwords * 4, 256);
  const size_t gap_b = f->gap ? align_up(nsub, 256) : 0;
  const size_t len_b = align_up(f->alphabet, 256);
  const size_t out_b = align_up(f->n * 2, 256);
  rc = ensure_stage(c, words_b + gap_b + len_b + out_b);
  if (rc) return rc;
  char* p = c->stage;
  hd_field d = *f;
  d.words = reinterpret_cast<const uint32_t*>(p);
  d.gap = f->gap ? reinterpret_cast<const uint8_t*>(p + words_b) : nullptr;
  d.lengths = reinterpret_cast<const uint8_t*>(p + words_b + gap_b);
  uint16_t* dout = reinterpret_cast<uint16_t*>(p + words_b + gap_b + len_b);
  if (cudaMemcpyAsync(p, f->words, f->nwords * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HD_ERR_CUDA;
  if (f->gap && cudaMemcpyAsync(p + words_b, f->gap, nsub, cudaMemcpyHostToDevice, st) !=
                    cudaSuccess)
    return HD_ERR_CUDA;
  if (cudaMemcpyAsync(p + words_b + gap_b, f->lengths, f->alphabet, cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return HD_ERR_CUDA;
  rc = decode_impl(c, &d, dout, nullptr, stream);
  if (rc) return rc;
  if (f->n && cudaMemcpyAsync(host_out, dout, f->n * 2, cudaMemcpyDeviceToHost, st) !=
                  cudaSuccess)
    return HD_ERR_CUDA;
  std::vector<uint32_t> bits;
  rc = read_errors(c, stream, bits);
  if (rc) return rc;
  if (c->host_status != HD_OK) return c->host_status;
  uint32_t all = 0;
  for (uint32_t b : bits) all |= b;
  return map_err_bits(all);
}

int hd_profile(hd_ctx* c, int enable) {
  if (!c) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->profile = enable != 0;
  return HD_OK;
}

int hd_kernel_time(hd_ctx* c, double* ms, uint64_t* launches) {
  if (!c || !ms || !launches) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  double total = 0;
  uint64_t n = 0;
  for (size_t k = 0; k + 1 < c->events_used; k += 2) {
    if (cudaEventSynchronize(c->events[k + 1]) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    float t = 0;
    if (cudaEventElapsedTime(&t, c->events[k], c->events[k + 1]) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    total += t;
    ++n;
  }
  c->events_used = 0;
  *ms = total;
  *launches = n;
  return HD_OK;
}

uint64_t hd_launch_count(hd_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
