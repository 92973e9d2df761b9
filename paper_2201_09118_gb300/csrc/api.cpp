// api.cpp -- the C ABI of hd.h: context, argument checks, workspace layout
// and the launch sequence (decode-table kernel, then the decode kernels of
// the field's strategy).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "hd.h"
#include "host_internal.h"
#include "kernels.h"

// Cached graph: strategy, launch shape, capacities and workspace address.
using GraphKey = std::tuple<bool, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t,
                            uint32_t, uint64_t, size_t, uintptr_t>;
// Autotuner class: strategy, mean code length in quarter bits, log2 of the
// symbol count, largest stream subsequence size of the batch.
using TuneKey = std::tuple<bool, uint32_t, uint32_t, uint32_t>;

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
  // per-phase timing while profiling: (phase, event before, event after)
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> phase_recs;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans;  // hd_kernel_time spans
  uint64_t launches = 0;
  hd::LaunchShape last_shape{};  // launch shape of the last decode
  // graph launches (hd_decode_batch)
  std::map<GraphKey, cudaGraphExec_t> graphs;
  cudaStream_t cap_stream = nullptr;  // capture only; graphs run on the caller's stream
  uint64_t captures = 0;
  char* pinned = nullptr;             // header + descriptors staged for the copy
  size_t pinned_cap = 0;
  cudaEvent_t pinned_ev = nullptr;
  bool pinned_busy = false;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};  // autotuner timing
  // pipelined host decode: copy streams, per-chunk events, pinned chunk ends
  cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
  std::vector<cudaEvent_t> pipe_ev;
  uint64_t* pin_ends = nullptr;      // host-mapped: chunk ends written by the tile scan
  uint64_t* pin_ends_dev = nullptr;  // the same memory as the device sees it
  uint64_t wait_limit = 0;           // one-pass decoder: cycles per look-back wait (0: default)
  // autotuner results: batch class -> launch shape
  std::map<TuneKey, hd_config> tuned;
  // Lorenzo reconstruction: its workspace (error word first), whether its
  // error word belongs to the last queued operation, decoded codes of
  // hd_decompress_device
  char* rws = nullptr;
  size_t rws_cap = 0;
  bool recon_active = false;
  uint16_t* dcodes = nullptr;
  size_t dcodes_cap = 0;
};

namespace {

using hd::FieldDesc;

constexpr uint32_t kDefaultThreads = 256;
// first-level table bits when the configuration leaves them open: 13 with
// 16-bit entries (alphabets up to 4096), else 12
constexpr double kRunsBelowBits = 4.0;  // mean code length below which counting uses runs
// mean code length below which runs of the 1-bit code are counted and written
// whole (long runs: measured 425 -> 660 GB/s at 1.01 bits per code, slower at
// 1.87 bits, whose runs are short)
constexpr double kZeroRunsBelowBits = 1.25;
constexpr uint32_t kDefaultK16 = 13;
constexpr uint32_t kTableSlices = 16;  // blocks building a single field's decode table
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

void drop_graphs(hd_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

int ensure_ws(hd_ctx* c, size_t bytes) {
  if (bytes <= c->ws_cap) return HD_OK;
  if (c->ws) {
    cudaDeviceSynchronize();
    drop_graphs(c);  // they hold addresses inside the old workspace
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

// Decoder subsequence when the configuration leaves it open: 256 bits (for
// gap arrays every second entry of a 128-bit stream's array), because the
// per-tile work of a thread then amortises its fixed costs better and, when
// synchronising, fewer boundaries have to be agreed on.
uint32_t default_decoder_S(uint32_t stream_S, bool gap) {
  if (!gap) return 256;
  return stream_S < 256 ? 256 : stream_S;
}

// A shape for the two-phase kernels (threads of one block = one tile of
// subsequences: 128, 256 or 512).
hd::LaunchShape two_phase_shape(hd::LaunchShape s) {
  if (s.threads != 128 && s.threads != 256 && s.threads != 512) s.threads = kDefaultThreads;
  s.decoder = 1;
  return s;
}

hd::LaunchShape shape_for(const hd_ctx* c, uint32_t stream_S, bool gap) {
  hd::LaunchShape s{};
  s.S = c->cfg.subseq_bits ? c->cfg.subseq_bits : default_decoder_S(stream_S, gap);
  s.threads = c->cfg.threads ? c->cfg.threads : kDefaultThreads;
  s.K = c->cfg.lut_bits;  // 0: chosen per launch
  s.window = c->cfg.window;  // 0: chosen per launch
  s.grid = 0;
  return two_phase_shape(s);
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

// Phases of hd_phase_times.
enum PhaseId { kPhSync = 0, kPhCount = 1, kPhIndex = 2, kPhWrite = 3 };

// Records an event on `st` that closes the phase opened by *open (when
// profiling) and opens the next one; returns the new event.
cudaEvent_t phase_mark(hd_ctx* c, cudaStream_t st, int phase, cudaEvent_t open) {
  cudaEvent_t e = next_event(c);
  cudaEventRecord(e, st);
  if (open) c->phase_recs.emplace_back(phase, open, e);
  return e;
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

uint64_t pow2_at_least(uint64_t v, uint64_t lo) {
  uint64_t p = lo;
  while (p < v) p <<= 1;
  return p;
}

// Workspace layout of one launch; [0, zero) is cleared by the table kernel.
struct Layout {
  size_t err = 0, zero = 0, hdr = 0, desc = 0, tab = 0, tile = 0, tbase = 0, count = 0;
  size_t gap = 0, ta = 0, te = 0, tf = 0, tg = 0, total = 0;
};

Layout make_layout(uint32_t nf, uint64_t tiles, uint64_t subs, size_t tab_bytes,
                   const hd::LaunchShape& s, bool self_sync, bool own_gap) {
  Layout L;
  size_t off = 0;
  L.err = off;
  off = align_up(off + 4ull * nf, 16);
  L.zero = off;
  L.hdr = align_up(off, 256);  // launch header, then the field descriptors
  L.desc = L.hdr + 256;
  off = L.desc + sizeof(FieldDesc) * nf;
  L.tab = align_up(off, 256);
  off = L.tab + tab_bytes;
  L.tile = align_up(off, 256);
  off = L.tile + 4ull * tiles;
  L.tbase = align_up(off, 256);  // exclusive scan of the tile totals
  off = L.tbase + 8ull * (tiles + 1);
  L.count = align_up(off, 256);
  off = L.count + hd::count_bytes_per_subsequence(s.S) * subs;
  // self-synchronisation: subsequence starts, tile links (16-byte padded)
  const size_t link_bytes = align_up(tiles + 1, 16) + 16;
  L.gap = align_up(off, 256);
  if (own_gap) off = L.gap + subs;
  L.ta = align_up(off, 256);
  L.te = align_up(L.ta + link_bytes, 256);
  L.tf = align_up(L.te + link_bytes, 256);
  L.tg = align_up(L.tf + tiles, 256);
  if (self_sync) off = L.tg + tiles;
  L.total = align_up(off, 256);
  return L;
}

// Host-side preparation of a launch: final shape, per-field tiles, counts
// and table offsets.
struct Prepared {
  hd::LaunchShape s;
  uint64_t tiles = 0, subs = 0;
  size_t tab_bytes = 0;
  std::vector<size_t> tab_off;  // relative to the table region
};

int prepare_launch(const hd_ctx* c, std::vector<FieldDesc>& descs, const hd::LaunchShape& shape,
                   bool self_sync, Prepared& P) {
  hd::LaunchShape s = shape;
  uint64_t bits = 0, syms = 0;
  uint32_t amax = 0;
  uint64_t syms_long = 0;  // symbols of fields of 4 or more bits per code
  for (auto& d : descs) {
    bits += d.nbits;
    syms += d.n;
    amax = std::max(amax, d.alphabet);
    if (static_cast<double>(d.nbits) >= kRunsBelowBits * static_cast<double>(d.n))
      syms_long += d.n;
  }
  const double bits_per = static_cast<double>(bits) / static_cast<double>(syms ? syms : 1);
  // symbols of codes longer than the first-level table, kept in shared memory
  s.long_cap = static_cast<uint32_t>(align_up(std::min<uint32_t>(amax, 4096), 8));
  if (s.K == 0) s.K = hd::lut16_usable(kDefaultK16, amax) ? kDefaultK16 : kDefaultK;
  // 16-bit first-level entries when every field's symbols fit 12 bits
  s.lut16 = hd::lut16_usable(s.K, amax) ? 1u : 0u;
  // run table for counting when codes are short (measured: +24% decode at
  // 1.9 bits per code, -6% at 9 bits); two codes per lookup in the
  // decode-and-write kernel when fields of 4+ bits per code hold under a
  // quarter of the launch's symbols (their prefixes rarely hold two codes, and
  // the batched workload, about half of them, decoded 3% slower with it);
  // fields under 1.25 bits write runs instead
  const uint32_t pairs = 4 * syms_long < syms ? hd::kShapePairs : 0u;
  s.runs = bits_per < kZeroRunsBelowBits ? 3u : bits_per < kRunsBelowBits ? (1u | pairs) : 0u;
  if (s.window == 0) {
    // output window: about 1.2x a tile's expected symbol count, rounded up to
    // a multiple of 2048 so that batches of similar code lengths share a shape
    const double want = 1.2 * s.threads * s.S / std::max(bits_per, 0.25) + 64.0;
    s.window = static_cast<uint32_t>(
        align_up(static_cast<size_t>(std::min(std::max(want, 1024.0), 16384.0)), 2048));
  }
  s.window = static_cast<uint32_t>(align_up(std::max(s.window, s.S), 8));
  // the window is an optimisation (larger outputs go through several
  // windows), so it shrinks to fit shared memory
  const size_t budget = static_cast<size_t>(c->max_smem) - 2048;
  while (s.window > std::max<uint32_t>(1024, s.S) && hd::two_phase_smem_bytes(s) > budget)
    s.window -= 512;
  if (hd::two_phase_smem_bytes(s) > budget) return HD_ERR_ARG;
  if (self_sync && hd::sync_smem_bytes(s) > budget) return HD_ERR_ARG;
  P.s = s;
  P.tiles = P.subs = 0;
  P.tab_bytes = 0;
  P.tab_off.resize(descs.size());
  for (size_t k = 0; k < descs.size(); ++k) {
    FieldDesc& d = descs[k];
    d.unit_begin = P.tiles;
    d.nunits = tiles_for(d.nsub, s);
    P.tiles += d.nunits;
    d.count_begin = P.subs;
    P.subs += d.nsub;
    P.tab_off[k] = P.tab_bytes;
    P.tab_bytes += hd::table_bytes(s.K, d.alphabet);
  }
  return HD_OK;
}

// Points every descriptor at its table, error word and (self-synchronisation)
// start array inside the workspace.
void bind_descs(std::vector<FieldDesc>& descs, char* ws, const Layout& L, const Prepared& P,
                bool self_sync, bool sync_only) {
  for (size_t k = 0; k < descs.size(); ++k) {
    FieldDesc& d = descs[k];
    d.table = reinterpret_cast<const hd::TableHeader*>(ws + L.tab + P.tab_off[k]);
    d.err = reinterpret_cast<uint32_t*>(ws + L.err) + k;
    if (self_sync) {
      if (!sync_only) d.gap_out = reinterpret_cast<uint8_t*>(ws + L.gap) + d.count_begin;
      d.gap = d.gap_out;
      d.gap_stride = 1;
    }
  }
}

// Kernel parameters of a launch.  `dyn`: sizes come from the device-side
// header, the parameters carry the capacities (graph launches).
void make_params(const std::vector<FieldDesc>& descs, char* ws, const Layout& L,
                 const hd::LaunchShape& s, bool self_sync, bool dyn, uint32_t nf_param,
                 uint64_t tiles_param, hd::PrepParams& pp, hd::DecodeParams& dp) {
  pp = hd::PrepParams{};
  pp.f0 = descs[0];
  pp.fields = reinterpret_cast<const FieldDesc*>(ws + L.desc);
  pp.hdr = dyn ? reinterpret_cast<const hd::LaunchHeader*>(ws + L.hdr) : nullptr;
  pp.nfields = nf_param;
  // a lone field's table is built by several blocks
  pp.slices = nf_param == 1 ? kTableSlices : 1u;
  pp.table_blocks = std::min<uint32_t>(nf_param * pp.slices, 1024);
  pp.K = s.K;
  pp.zero_ptr = reinterpret_cast<uint4*>(ws);
  pp.zero_vec = L.zero / 16;
  pp.zero_blocks = static_cast<uint32_t>(std::min<uint64_t>((pp.zero_vec + 4095) / 4096, 64));
  if (pp.zero_blocks == 0) pp.zero_blocks = 1;
  dp = hd::DecodeParams{};
  dp.f0 = descs[0];
  dp.fields = pp.fields;
  dp.hdr = pp.hdr;
  dp.nfields = nf_param;
  dp.K = s.K;
  dp.window = s.window;
  dp.long_cap = s.long_cap;
  dp.zero_runs = (s.runs >> 1) & 1u;
  dp.total_units = tiles_param;
  dp.counts = ws + L.count;
  dp.tile_total = reinterpret_cast<uint32_t*>(ws + L.tile);
  dp.tile_base = reinterpret_cast<uint64_t*>(ws + L.tbase);
  if (self_sync) {
    dp.tile_a = reinterpret_cast<uint8_t*>(ws + L.ta);
    dp.tile_e = reinterpret_cast<uint8_t*>(ws + L.te);
    dp.tile_flag = reinterpret_cast<uint8_t*>(ws + L.tf);
    dp.tile_guess = reinterpret_cast<uint8_t*>(ws + L.tg);
  }
}

// The kernels of one strategy, in stream order:
//   gap array            table kernel, count kernel, tile scan, decode-and-write
//                        kernel;
//   self-synchronisation table kernel, synchronising kernel, link-fix kernel,
//                        then the same tile scan and decode-and-write kernel
//                        (with sync_only the last two are left out: the starts
//                        stay in each gap_out).
cudaError_t launch_all(const hd_ctx* c, const hd::PrepParams& pp, const hd::DecodeParams& dp,
                       const hd::LaunchShape& s, bool self_sync, bool sync_only,
                       cudaStream_t st) {
  cudaError_t e = hd::launch_prepare(pp, st);
  if (e != cudaSuccess) return e;
  if (self_sync) {
    e = hd::launch_sync(dp, s, c->num_sms, st);
    if (e == cudaSuccess && !sync_only) e = hd::launch_write(dp, s, c->num_sms, st);
    return e;
  }
  return hd::launch_decode_two_phase(dp, s, c->num_sms, st);
}

uint32_t kernels_per_launch(bool self_sync, bool sync_only) {
  return self_sync ? (sync_only ? 4u : 6u) : 4u;
}

// Gap-array decode with per-tile compression-ratio classes (Sec. IV-C,
// Algorithm 2): count and scan as usual, sort the tiles into classes by
// codeword count on the GPU, read the class sizes back (the paper also
// returns its class histogram to the host), then one decode-and-write launch
// per non-empty class with a window for that class: class c (compression
// ratio in (c, c+1], i.e. up to (c+1) * B * S / 16 codewords per tile) gets
// that many symbols, the last class the largest window shared memory holds.
int queue_cr_classes(hd_ctx* c, hd::DecodeParams dp, const Prepared& P, char* cls,
                     uint32_t nclass, cudaStream_t st) {
  uint32_t* counts = reinterpret_cast<uint32_t*>(cls);
  uint32_t* lists = reinterpret_cast<uint32_t*>(cls + 256);
  const uint64_t cap = P.tiles;
  const uint32_t unit = P.s.threads * P.s.S / 16;
  if (hd::launch_phase(dp, P.s, hd::Phase::kCount, c->num_sms, st) != cudaSuccess ||
      hd::launch_phase(dp, P.s, hd::Phase::kScan, c->num_sms, st) != cudaSuccess ||
      cudaMemsetAsync(counts, 0, 4ull * nclass, st) != cudaSuccess ||
      hd::launch_classify(dp, unit, nclass, counts, lists, cap, st) != cudaSuccess)
    return HD_ERR_CUDA;
  std::vector<uint32_t> n_in(nclass);
  if (cudaMemcpyAsync(n_in.data(), counts, 4ull * nclass, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  c->launches += 3;
  const size_t budget = static_cast<size_t>(c->max_smem) - 2048;
  for (uint32_t k = 0; k < nclass; ++k) {
    if (!n_in[k]) continue;
    hd::LaunchShape sh = P.s;
    uint64_t want = static_cast<uint64_t>(k + 1) * unit;
    if (k + 1 == nclass) want = 1ull << 20;
    sh.window = static_cast<uint32_t>(align_up(std::max<uint64_t>(want, sh.S), 8));
    sh.window = std::min<uint32_t>(sh.window, 1u << 20);
    while (sh.window > std::max<uint32_t>(1024, sh.S) && hd::two_phase_smem_bytes(sh) > budget)
      sh.window = sh.window > 4096 ? sh.window - 2048 : sh.window - 512;
    if (hd::two_phase_smem_bytes(sh) > budget) return HD_ERR_ARG;
    hd::DecodeParams d = dp;
    d.window = sh.window;
    d.tile_list = lists + k * cap;
    d.unit_lo = 0;
    d.unit_hi = n_in[k];
    if (hd::launch_phase(d, sh, hd::Phase::kWrite, c->num_sms, st) != cudaSuccess)
      return HD_ERR_CUDA;
    c->launches += 1;
  }
  return HD_OK;
}

// Decode + 1D Lorenzo reconstruction: where the values go and the outliers.
struct ValueArgs {
  float* vout;
  int32_t radius;
  float ebx2;
  const uint64_t* out_idx;
  const int32_t* out_val;
  uint64_t n_out;
  uint32_t* verr;  // error word of the reconstruction (cleared by the caller)
};

// Queues a decode of fields that all use the same strategy with direct
// kernel launches (sizes as kernel parameters).  With `va` (one gap-array
// field): values instead of codes.
// Time limit of one look-back wait of the one-pass decoder (SM clock cycles,
// about 2 s at GB300 clocks); a wait that runs out reports HD_ERR_TIMEOUT.
constexpr uint64_t kLookbackTimeoutCycles = 4000000000ull;

// Column symbols per lane of the one-pass decoder for a field of `bits_per`
// bits per code: about 1.3x a subsequence's expected codeword count, even.
uint32_t one_pass_cmax(uint32_t S, double bits_per) {
  const double want = 1.3 * S / std::max(bits_per, 0.25) + 2.0;
  uint32_t c = static_cast<uint32_t>(std::ceil(want));
  c = (c + 1) & ~1u;
  return std::min<uint32_t>(std::max<uint32_t>(c, 4), std::min<uint32_t>(S, 512));
}

// Queues a one-pass decode of one gap-array field (decode_warp.cu).
// Workspace: error word | abort flag | one look-back state per tile
// (the three cleared by the table kernel) | decode table.
int queue_decode_one_pass(hd_ctx* c, std::vector<FieldDesc>& descs, const hd::LaunchShape& shape,
                          cudaStream_t st) {
  FieldDesc& d = descs[0];
  hd::LaunchShape s = shape;
  const double bits_per =
      static_cast<double>(d.nbits) / static_cast<double>(d.n ? d.n : 1);
  if (s.K == 0) s.K = hd::lut16_usable(kDefaultK16, d.alphabet) ? kDefaultK16 : kDefaultK;
  // long-code symbols in shared memory (codes past the second-level tables);
  // none with 14+ table bits, whose first-level table takes that room
  s.long_cap = s.K >= 14 ? 0u
                         : static_cast<uint32_t>(align_up(std::min<uint32_t>(d.alphabet, 4096), 8));
  s.lut16 = hd::lut16_usable(s.K, d.alphabet) ? 1u : 0u;
  s.runs = 0;
  s.decoder = 2;
  s.cmax = one_pass_cmax(s.S, bits_per);
  s.window = 32 * s.cmax;
  const size_t budget = static_cast<size_t>(c->max_smem) - 2048;
  const bool fixed_threads = s.threads != 0;
  if (!fixed_threads) {
    // the most warps per block that shared memory holds
    for (uint32_t b : {1024u, 768u, 512u, 256u, 128u}) {
      s.threads = b;
      if (hd::warp_decode_smem_bytes(s) <= budget) break;
    }
  }
  if (s.threads != 128 && s.threads != 256 && s.threads != 512 && s.threads != 768 &&
      s.threads != 1024)
    return HD_ERR_ARG;
  // the column is an optimisation (overflowing lanes decode again), so it
  // shrinks to fit shared memory
  while (s.cmax > 4 && hd::warp_decode_smem_bytes(s) > budget) s.cmax -= 2;
  s.window = 32 * s.cmax;
  if (hd::warp_decode_smem_bytes(s) > budget) return HD_ERR_ARG;
  d.unit_begin = 0;
  d.nunits = (d.nsub + 31) / 32;
  d.count_begin = 0;
  const size_t tk_off = 16, st_off = 32;
  const size_t zero = align_up(st_off + 8 * d.nunits, 16);
  const size_t tab_off = align_up(zero, 256);
  const size_t need = tab_off + hd::table_bytes(s.K, d.alphabet);
  int rc = ensure_ws(c, need);
  if (rc) return rc;
  char* ws = c->ws;
  d.table = reinterpret_cast<const hd::TableHeader*>(ws + tab_off);
  d.err = reinterpret_cast<uint32_t*>(ws);
  hd::PrepParams pp{};
  pp.f0 = d;
  pp.nfields = 1;
  pp.slices = kTableSlices;
  pp.table_blocks = kTableSlices;
  pp.K = s.K;
  pp.zero_ptr = reinterpret_cast<uint4*>(ws);
  pp.zero_vec = zero / 16;
  pp.zero_blocks = static_cast<uint32_t>(std::min<uint64_t>((pp.zero_vec + 4095) / 4096, 64));
  if (pp.zero_blocks == 0) pp.zero_blocks = 1;
  hd::DecodeParams dp{};
  dp.f0 = d;
  dp.nfields = 1;
  dp.K = s.K;
  dp.window = s.window;
  dp.cmax = s.cmax;
  dp.long_cap = s.long_cap;
  dp.total_units = d.nunits;
  dp.unit_state = reinterpret_cast<uint64_t*>(ws + st_off);
  dp.ticket = reinterpret_cast<uint32_t*>(ws + tk_off);
  dp.abort_flag = reinterpret_cast<uint32_t*>(ws + tk_off) + 1;
  dp.timeout_cycles = c->wait_limit ? c->wait_limit : kLookbackTimeoutCycles;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    e0 = next_event(c);
    e1 = next_event(c);
  }
  cudaError_t e = hd::launch_prepare(pp, st);
  if (e == cudaSuccess && c->profile) cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = hd::launch_decode_warp(dp, s, c->num_sms, st);
  if (c->profile) {
    cudaEventRecord(e1, st);
    c->spans.emplace_back(e0, e1);
    c->phase_recs.emplace_back(kPhWrite, e0, e1);  // one kernel does every phase
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  c->launches += 2;
  c->err_off = 0;
  c->err_count = 1;
  c->recon_active = false;
  c->last_shape = s;
  return HD_OK;
}

int queue_decode(hd_ctx* c, std::vector<FieldDesc>& descs, const hd::LaunchShape& shape_in,
                 bool self_sync, bool sync_only, cudaStream_t st,
                 const ValueArgs* va = nullptr) {
  const uint32_t nf = static_cast<uint32_t>(descs.size());
  if (!self_sync && !sync_only && !va && nf == 1 && shape_in.decoder == 2 && !c->cfg.cr_classes)
    return queue_decode_one_pass(c, descs, shape_in, st);
  const hd::LaunchShape shape = two_phase_shape(shape_in);
  Prepared P;
  int rc = prepare_launch(c, descs, shape, self_sync, P);
  if (rc) return rc;
  const Layout L = make_layout(nf, P.tiles, P.subs, P.tab_bytes, P.s, self_sync,
                               self_sync && !sync_only);
  const uint32_t nclass = self_sync || va ? 0u : c->cfg.cr_classes;
  const size_t cls_off = L.total;  // CR classes: counts, then one tile list per class
  const size_t cls_bytes = nclass ? 256 + 4ull * nclass * P.tiles : 0;
  // values: tile residue sums, q bases, outlier bases, outlier corrections
  const size_t rs_off = align_up(L.total, 256);
  const size_t qb_off = align_up(rs_off + 4ull * P.tiles, 256);
  const size_t ob_off = align_up(qb_off + 8ull * (P.tiles + 1), 256);
  const size_t co_off = align_up(ob_off + 8ull * (P.tiles + 1), 256);
  const size_t need = va ? co_off + 4ull * (va->n_out + 1) : L.total + cls_bytes;
  rc = ensure_ws(c, need);
  if (rc) return rc;
  char* ws = c->ws;
  bind_descs(descs, ws, L, P, self_sync, sync_only);
  if (nf > 1 && cudaMemcpyAsync(ws + L.desc, descs.data(), sizeof(FieldDesc) * nf,
                                cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HD_ERR_CUDA;
  hd::PrepParams pp;
  hd::DecodeParams dp;
  make_params(descs, ws, L, P.s, self_sync, false, nf, P.tiles, pp, dp);
  if (va) {
    dp.tile_rsum = reinterpret_cast<uint32_t*>(ws + rs_off);
    dp.tile_qbase = reinterpret_cast<uint64_t*>(ws + qb_off);
    dp.tile_obase = reinterpret_cast<uint64_t*>(ws + ob_off);
    dp.out_corr = reinterpret_cast<const int32_t*>(ws + co_off);
    dp.vout = va->vout;
    dp.radius = va->radius;
    dp.ebx2 = va->ebx2;
    dp.out_idx = va->out_idx;
    dp.out_val = va->out_val;
    dp.n_out = va->n_out;
    dp.verr = va->verr;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    e0 = next_event(c);
    e1 = next_event(c);
  }
  // the timed span starts after the table kernel
  cudaError_t e = hd::launch_prepare(pp, st);
  if (e == cudaSuccess && c->profile) cudaEventRecord(e0, st);
  if (e == cudaSuccess && c->profile && !va && !nclass) {
    // the same kernels one phase at a time, with an event between phases
    cudaEvent_t m = e0;
    if (self_sync) {
      e = hd::launch_sync(dp, P.s, c->num_sms, st);
      m = phase_mark(c, st, kPhSync, m);
    } else {
      e = hd::launch_phase(dp, P.s, hd::Phase::kCount, c->num_sms, st);
      m = phase_mark(c, st, kPhCount, m);
    }
    if (e == cudaSuccess && !sync_only) {
      e = hd::launch_phase(dp, P.s, hd::Phase::kScan, c->num_sms, st);
      m = phase_mark(c, st, kPhIndex, m);
      if (e == cudaSuccess) e = hd::launch_phase(dp, P.s, hd::Phase::kWrite, c->num_sms, st);
      m = phase_mark(c, st, kPhWrite, m);
    }
  } else if (e == cudaSuccess) {
    if (self_sync) {
      e = hd::launch_sync(dp, P.s, c->num_sms, st);
      if (e == cudaSuccess && !sync_only) e = hd::launch_write(dp, P.s, c->num_sms, st);
    } else if (va) {
      e = hd::launch_outlier_prefix(va->out_val, va->n_out, va->radius,
                                    reinterpret_cast<int32_t*>(ws + co_off), st);
      if (e == cudaSuccess) e = hd::launch_decode_values(dp, P.s, c->num_sms, st);
    } else if (nclass) {
      rc = queue_cr_classes(c, dp, P, ws + cls_off, nclass, st);
      if (rc) return rc;
    } else {
      e = hd::launch_decode_two_phase(dp, P.s, c->num_sms, st);
    }
  }
  if (c->profile) {
    cudaEventRecord(e1, st);
    c->spans.emplace_back(e0, e1);
  }
  if (e != cudaSuccess) return HD_ERR_CUDA;
  c->launches += kernels_per_launch(self_sync, sync_only) + (va ? 2 : 0);
  c->err_off = L.err;
  c->err_count = nf;
  c->recon_active = false;
  c->last_shape = P.s;
  return HD_OK;
}

// Queues the same work as one CUDA graph launch.  The graph is captured once
// per (strategy, launch shape, capacity class) and replayed for every later
// batch that fits: field and tile counts travel in the device-side launch
// header and the descriptors, both copied in before the replay from pinned
// host memory.  Capacities are powers of two, so a context holds few graphs.
int queue_decode_graph(hd_ctx* c, std::vector<FieldDesc>& descs, const hd::LaunchShape& shape_in,
                       bool self_sync, cudaStream_t st) {
  const uint32_t nf = static_cast<uint32_t>(descs.size());
  const hd::LaunchShape shape = two_phase_shape(shape_in);
  Prepared P;
  int rc = prepare_launch(c, descs, shape, self_sync, P);
  if (rc) return rc;
  const uint32_t cap_f = static_cast<uint32_t>(pow2_at_least(nf, 16));
  const uint64_t cap_t = pow2_at_least(P.tiles, 1024);
  const uint64_t cap_s = cap_t * P.s.threads;
  const size_t cap_tab = static_cast<size_t>(pow2_at_least(P.tab_bytes, 1 << 16));
  const Layout L = make_layout(cap_f, cap_t, cap_s, cap_tab, P.s, self_sync, self_sync);
  rc = ensure_ws(c, L.total);
  if (rc) return rc;
  char* ws = c->ws;
  bind_descs(descs, ws, L, P, self_sync, false);

  // header + descriptors through pinned memory (wait until the previous copy
  // out of it has run before overwriting it)
  const size_t stage_bytes = 256 + sizeof(FieldDesc) * nf;
  if (c->pinned_busy) {
    if (cudaEventSynchronize(c->pinned_ev) != cudaSuccess) return HD_ERR_CUDA;
    c->pinned_busy = false;
  }
  if (stage_bytes > c->pinned_cap) {
    if (c->pinned) cudaFreeHost(c->pinned);
    c->pinned = nullptr;
    c->pinned_cap = 0;
    const size_t cap = align_up(std::max<size_t>(stage_bytes, 64 << 10), 64 << 10);
    if (cudaMallocHost(&c->pinned, cap) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_NOMEM;
    }
    c->pinned_cap = cap;
  }
  hd::LaunchHeader h{};
  h.total_units = P.tiles;
  h.nfields = nf;
  std::memset(c->pinned, 0, 256);
  std::memcpy(c->pinned, &h, sizeof(h));
  std::memcpy(c->pinned + 256, descs.data(), sizeof(FieldDesc) * nf);
  if (cudaMemcpyAsync(ws + L.hdr, c->pinned, stage_bytes, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaEventRecord(c->pinned_ev, st) != cudaSuccess)
    return HD_ERR_CUDA;
  c->pinned_busy = true;

  const GraphKey key{self_sync, P.s.S,     P.s.threads, P.s.K, P.s.window, P.s.long_cap,
                     P.s.lut16 | (P.s.runs << 1), cap_f, cap_t, cap_tab,
                     reinterpret_cast<uintptr_t>(ws)};
  auto it = c->graphs.find(key);
  cudaGraphExec_t exec = nullptr;
  if (it != c->graphs.end()) {
    exec = it->second;
  } else {
    hd::PrepParams pp;
    hd::DecodeParams dp;
    make_params(descs, ws, L, P.s, self_sync, true, cap_f, cap_t, pp, dp);
    if (!c->cap_stream &&
        cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return HD_ERR_CUDA;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return HD_ERR_CUDA;
    const cudaError_t le = launch_all(c, pp, dp, P.s, self_sync, false, c->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    c->graphs.emplace(key, exec);
    c->captures += 1;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    e0 = next_event(c);
    e1 = next_event(c);
    cudaEventRecord(e0, st);
  }
  const cudaError_t e = cudaGraphLaunch(exec, st);
  if (c->profile) {
    cudaEventRecord(e1, st);
    c->spans.emplace_back(e0, e1);
  }
  if (e != cudaSuccess) return HD_ERR_CUDA;
  c->launches += kernels_per_launch(self_sync, false);
  c->err_off = L.err;
  c->err_count = nf;
  c->recon_active = false;
  c->last_shape = P.s;
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


TuneKey tune_key(bool gap, uint32_t maxS, uint64_t bits, uint64_t syms) {
  const double mean = static_cast<double>(bits) / static_cast<double>(syms ? syms : 1);
  uint32_t lg = 0;
  while ((1ull << (lg + 1)) <= syms) ++lg;
  return TuneKey{!gap, static_cast<uint32_t>(mean * 4.0), lg, maxS};
}

// Launch shape of one strategy group of a batch: the context's configuration,
// else the autotuned shape of the group's class, else the defaults.
hd::LaunchShape group_shape(const hd_ctx* c, const hd_field* fs, const std::vector<uint32_t>& idx,
                            bool gap) {
  uint32_t maxS = 0;
  uint64_t bits = 0, syms = 0;
  for (uint32_t i : idx) {
    maxS = std::max(maxS, fs[i].subseq_bits);
    bits += fs[i].nbits;
    syms += fs[i].n;
  }
  const hd_config& k = c->cfg;
  const bool user =
      k.subseq_bits || k.threads || k.window || k.lut_bits || k.cr_classes || k.decoder;
  hd_config use = k;
  if (!user) {
    auto it = c->tuned.find(tune_key(gap, maxS, bits, syms));
    if (it != c->tuned.end()) use = it->second;
  }
  hd::LaunchShape s{};
  s.S = use.subseq_bits ? use.subseq_bits : default_decoder_S(maxS ? maxS : 128, gap);
  if (!gap && s.S > 256) s.S = 256;
  s.threads = use.threads;  // 0: chosen per launch
  s.K = use.lut_bits;  // 0: chosen per launch
  s.window = use.window;
  // one pass decodes single gap-array fields; groups of several fields and
  // self-synchronisation run the two-phase kernels
  s.decoder = gap && idx.size() == 1 && use.decoder != 1 && !use.cr_classes ? 2u : 1u;
  if (s.decoder == 1) s = two_phase_shape(s);
  return s;
}

// Launch shape of a single-field decode: as for a batch of that one field.
hd::LaunchShape field_shape(const hd_ctx* c, const hd_field* f, bool gap) {
  const std::vector<uint32_t> one{0};
  return group_shape(c, f, one, gap);
}

struct BatchPlan {
  std::vector<uint32_t> gap_i, sync_i;  // fields with work, by strategy
};

// Sorts the fields of a batch into the two strategy groups; fields with
// nothing to decode (n == 0 and nbits == 0) are left out.
int plan_batch(hd_ctx* c, const hd_field* fs, uint32_t nf, uint16_t* const* d_outs,
               BatchPlan& plan) {
  (void)c;
  (void)d_outs;
  for (uint32_t i = 0; i < nf; ++i) {
    const hd_field* f = &fs[i];
    if (f->n == 0 && f->nbits == 0) continue;
    if (f->nbits == 0 || f->n == 0) return HD_ERR_CORRUPT;
    (f->gap ? plan.gap_i : plan.sync_i).push_back(i);
  }
  return HD_OK;
}

// hd_decode_batch with the context lock held.  Each strategy group is one
// graph launch; with both groups present the first group's error words are
// read before the second reuses the workspace.
int decode_batch_locked(hd_ctx* c, const hd_field* fs, uint32_t nf, uint16_t* const* d_outs,
                        void* stream) {
  c->err_count = 0;
  c->recon_active = false;
  c->host_status = HD_OK;
  c->err_map.assign(nf, 0xffffffffu);
  if (nf == 0) return HD_OK;
  for (uint32_t i = 0; i < nf; ++i) {
    const int rc = check_field(&fs[i], true, d_outs[i]);
    if (rc == HD_PENDING) continue;
    if (rc) {
      c->host_status = rc;
      return rc;
    }
  }
  BatchPlan plan;
  int rc = plan_batch(c, fs, nf, d_outs, plan);
  if (rc == HD_ERR_CORRUPT) {
    c->host_status = HD_ERR_CORRUPT;  // symbols without bits or bits without symbols
    return HD_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool both = !plan.gap_i.empty() && !plan.sync_i.empty();
  std::vector<uint32_t> merged(nf, 0);
  for (int grp = 0; grp < 2; ++grp) {
    const bool ss = grp == 1;
    const std::vector<uint32_t>& idx = ss ? plan.sync_i : plan.gap_i;
    if (idx.empty()) continue;
    const hd::LaunchShape s = group_shape(c, fs, idx, !ss);
    std::vector<FieldDesc> d;
    d.reserve(idx.size());
    for (uint32_t i : idx) {
      if (!ss && s.S % fs[i].subseq_bits) {
        c->host_status = HD_ERR_ARG;
        return HD_ERR_ARG;
      }
      FieldDesc x;
      fill_desc(x, &fs[i], s, d_outs[i]);
      d.push_back(x);
    }
    rc = queue_decode_graph(c, d, s, ss, st);
    if (rc) {
      c->host_status = rc;
      return rc;
    }
    if (!both) {
      for (size_t k = 0; k < idx.size(); ++k) c->err_map[idx[k]] = static_cast<uint32_t>(k);
      return HD_OK;
    }
    std::vector<uint32_t> bits;
    rc = read_errors(c, stream, bits);
    if (rc) return rc;
    for (size_t k = 0; k < idx.size(); ++k) merged[idx[k]] = bits[k];
  }
  // both groups ran: the per-field results are kept on the host
  c->err_count = 0;
  c->recon_active = false;
  for (uint32_t i = 0; i < nf; ++i) c->err_map[i] = 0x80000000u | merged[i];
  return HD_OK;
}


constexpr uint32_t kMaxChunks = 16;

// hd_decode_host for a large gap-array field as a copy/decode pipeline (the
// host-to-device transfer is part of the paper's end-to-end comparison,
// Sec. V): the stream is copied to the device in chunks of whole tiles on one
// copy stream, each chunk is counted, scanned and decoded on the caller's
// stream as soon as its bits have arrived, and its symbols go back to the host
// on a second copy stream as soon as they are written.  The host learns where
// a chunk's symbols end from its tile scan (one 8-byte read per chunk), so the
// three directions overlap.  Context lock held; `f` holds host pointers.
int decode_host_pipelined(hd_ctx* c, const hd_field* f, uint16_t* host_out, cudaStream_t st,
                          bool* used) {
  *used = false;
  const uint64_t nsub_stream = (f->nbits + f->subseq_bits - 1) / f->subseq_bits;
  const size_t words_b = align_up(f->nwords * 4, 256);
  const size_t gap_b = align_up(nsub_stream, 256);
  const size_t len_b = align_up(f->alphabet, 256);
  const size_t out_b = align_up(f->n * 2, 256);
  hd_field d = *f;  // device copy of the field, pointers into the staging area
  hd::LaunchShape shape = two_phase_shape(field_shape(c, &d, true));
  if (shape.S % f->subseq_bits) return HD_OK;  // not pipelined
  std::vector<FieldDesc> descs(1);
  {
    int rc = ensure_stage(c, words_b + gap_b + len_b + out_b);
    if (rc) return rc;
  }
  char* p = c->stage;
  d.words = reinterpret_cast<const uint32_t*>(p);
  d.gap = reinterpret_cast<const uint8_t*>(p + words_b);
  d.lengths = reinterpret_cast<const uint8_t*>(p + words_b + gap_b);
  uint16_t* dout = reinterpret_cast<uint16_t*>(p + words_b + gap_b + len_b);
  fill_desc(descs[0], &d, shape, dout);
  Prepared P;
  int rc = prepare_launch(c, descs, shape, false, P);
  if (rc) return rc;
  if (P.tiles < 4ull * c->num_sms) return HD_OK;  // too small to pipeline
  const Layout L = make_layout(1, P.tiles, P.subs, P.tab_bytes, P.s, false, false);
  rc = ensure_ws(c, L.total);
  if (rc) return rc;
  char* ws = c->ws;
  bind_descs(descs, ws, L, P, false, false);
  hd::PrepParams pp;
  hd::DecodeParams dp;
  make_params(descs, ws, L, P.s, false, false, 1, P.tiles, pp, dp);
  if (!c->s_h2d && cudaStreamCreateWithFlags(&c->s_h2d, cudaStreamNonBlocking) != cudaSuccess)
    return HD_ERR_CUDA;
  if (!c->s_d2h && cudaStreamCreateWithFlags(&c->s_d2h, cudaStreamNonBlocking) != cudaSuccess)
    return HD_ERR_CUDA;
  while (c->pipe_ev.size() < 3 * kMaxChunks + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HD_ERR_CUDA;
    c->pipe_ev.push_back(e);
  }
  if (!c->pin_ends) {
    void* hp = nullptr;
    void* dptr = nullptr;
    if (cudaHostAlloc(&hp, 8 * kMaxChunks, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_NOMEM;
    }
    if (cudaHostGetDevicePointer(&dptr, hp, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(hp);
      return HD_ERR_CUDA;
    }
    c->pin_ends = static_cast<uint64_t*>(hp);
    c->pin_ends_dev = static_cast<uint64_t*>(dptr);
  }
  *used = true;
  const uint64_t units_per_sub = P.s.S / 32;
  const uint64_t tiles = P.tiles;
  const uint32_t nch = static_cast<uint32_t>(
      std::min<uint64_t>(kMaxChunks, std::max<uint64_t>(1, tiles / (2ull * c->num_sms))));
  const uint64_t per = (tiles + nch - 1) / nch;
  cudaEvent_t* ev_in = c->pipe_ev.data();
  cudaEvent_t* ev_end = ev_in + kMaxChunks;
  cudaEvent_t* ev_out = ev_end + kMaxChunks;
  cudaEvent_t ev_done = ev_out[kMaxChunks];
  // lengths and the whole gap array (small) first, then the decode tables
  if (cudaMemcpyAsync(p + words_b + gap_b, f->lengths, f->alphabet, cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(p + words_b, f->gap, nsub_stream, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      hd::launch_prepare(pp, st) != cudaSuccess)
    return HD_ERR_CUDA;
  c->launches += 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    e0 = next_event(c);
    e1 = next_event(c);
    cudaEventRecord(e0, st);
  }
  for (uint32_t j = 0; j < nch; ++j) {
    const uint64_t t0 = j * per, t1 = std::min<uint64_t>(tiles, t0 + per);
    // units of the chunk's subsequences plus the one a codeword near the end
    // may reach
    const uint64_t w0 = t0 * P.s.threads * units_per_sub;
    const uint64_t w1 = std::min<uint64_t>(f->nwords, t1 * P.s.threads * units_per_sub + 1);
    if (w1 > w0 && cudaMemcpyAsync(p + 4 * w0, f->words + w0, 4 * (w1 - w0),
                                   cudaMemcpyHostToDevice, c->s_h2d) != cudaSuccess)
      return HD_ERR_CUDA;
    if (cudaEventRecord(ev_in[j], c->s_h2d) != cudaSuccess ||
        cudaStreamWaitEvent(st, ev_in[j], 0) != cudaSuccess)
      return HD_ERR_CUDA;
    dp.unit_lo = t0;
    dp.unit_hi = t1;
    dp.scan_end = c->pin_ends_dev + j;  // the scan stores the chunk's end for the host
    if (hd::launch_phase(dp, P.s, hd::Phase::kCount, c->num_sms, st) != cudaSuccess ||
        hd::launch_phase(dp, P.s, hd::Phase::kScan, c->num_sms, st) != cudaSuccess ||
        cudaEventRecord(ev_end[j], st) != cudaSuccess ||
        hd::launch_phase(dp, P.s, hd::Phase::kWrite, c->num_sms, st) != cudaSuccess ||
        cudaEventRecord(ev_out[j], st) != cudaSuccess)
      return HD_ERR_CUDA;
    c->launches += 3;
  }
  if (c->profile) {
    cudaEventRecord(e1, st);
    c->spans.emplace_back(e0, e1);
  }
  // symbols back to the host, chunk by chunk, as their ends become known
  uint64_t done = 0;
  for (uint32_t j = 0; j < nch; ++j) {
    if (cudaEventSynchronize(ev_end[j]) != cudaSuccess) return HD_ERR_CUDA;
    const uint64_t chunk_end = *const_cast<volatile uint64_t*>(c->pin_ends + j);
    const uint64_t end = std::min<uint64_t>(f->n, chunk_end);
    if (end > done) {
      if (cudaStreamWaitEvent(c->s_d2h, ev_out[j], 0) != cudaSuccess ||
          cudaMemcpyAsync(host_out + done, dout + done, 2 * (end - done), cudaMemcpyDeviceToHost,
                          c->s_d2h) != cudaSuccess)
        return HD_ERR_CUDA;
      done = end;
    }
  }
  if (cudaEventRecord(ev_done, c->s_d2h) != cudaSuccess ||
      cudaStreamWaitEvent(st, ev_done, 0) != cudaSuccess)
    return HD_ERR_CUDA;
  c->err_off = L.err;
  c->err_count = 1;
  c->recon_active = false;
  c->host_status = HD_OK;
  c->last_shape = P.s;
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
          cudaSuccess ||
      cudaEventCreateWithFlags(&c->pinned_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&c->tune_ev[0]) != cudaSuccess ||
      cudaEventCreate(&c->tune_ev[1]) != cudaSuccess) {
    cudaGetLastError();
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
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->pinned_ev) cudaEventDestroy(c->pinned_ev);
    if (c->s_h2d) cudaStreamDestroy(c->s_h2d);
    if (c->s_d2h) cudaStreamDestroy(c->s_d2h);
    for (auto e : c->pipe_ev) cudaEventDestroy(e);
    if (c->pin_ends) cudaFreeHost(c->pin_ends);  // cudaHostAlloc memory
    for (auto e : c->tune_ev)
      if (e) cudaEventDestroy(e);
    if (c->ws) cudaFree(c->ws);
    if (c->stage) cudaFree(c->stage);
    if (c->rws) cudaFree(c->rws);
    if (c->dcodes) cudaFree(c->dcodes);
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
  if (cfg->decoder > 2) return HD_ERR_ARG;
  if (cfg->threads && cfg->threads != 128 && cfg->threads != 256 && cfg->threads != 512 &&
      !((cfg->threads == 768 || cfg->threads == 1024) && cfg->decoder == 2))
    return HD_ERR_ARG;
  if (cfg->lut_bits && (cfg->lut_bits < 8 || cfg->lut_bits > 15)) return HD_ERR_ARG;
  if (cfg->cr_classes && (cfg->cr_classes < 2 || cfg->cr_classes > 32)) return HD_ERR_ARG;
  if (cfg->window && (cfg->window < 64 || cfg->window > 32768)) return HD_ERR_ARG;
  c->cfg = *cfg;
  return HD_OK;
}

int hd_get_config(hd_ctx* c, hd_config* cfg) {
  if (!c || !cfg) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  cfg->subseq_bits = c->cfg.subseq_bits ? c->cfg.subseq_bits : c->last_shape.S;
  cfg->threads = c->cfg.threads ? c->cfg.threads
                 : c->last_shape.threads ? c->last_shape.threads : kDefaultThreads;
  cfg->window = c->cfg.window ? c->cfg.window : c->last_shape.window;
  cfg->lut_bits = c->cfg.lut_bits ? c->cfg.lut_bits : c->last_shape.K;
  cfg->cr_classes = c->cfg.cr_classes;
  cfg->decoder = c->cfg.decoder ? c->cfg.decoder : c->last_shape.decoder;
  return HD_OK;
}

static int decode_impl(hd_ctx* c, const hd_field* f, uint16_t* d_out, uint8_t* gap_out,
                       void* stream) {
  const bool sync_only = gap_out != nullptr;
  int rc = check_field(f, !sync_only, d_out);
  c->err_count = 0;
  c->recon_active = false;
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
  hd::LaunchShape s = sync_only ? shape_for(c, f->subseq_bits, false)
                                : field_shape(c, f, !self_sync);
  if (self_sync && s.S > 256) s.S = 256;  // the synchronising kernel stops at 256-bit subsequences
  if (sync_only) s.S = f->subseq_bits;    // one gap entry per stream subsequence
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

int hd_inspect_tables(hd_ctx* c, const uint8_t* lengths, uint32_t alphabet, uint32_t K,
                      uint16_t* lut16, uint8_t* len8, uint8_t* run8, uint32_t* pair,
                      void* stream) {
  if (!c || !lengths || alphabet < 2 || alphabet > 4096 || K < 8 || K > 15) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // error word | table, in a buffer of its own (the context's workspace may
  // still be in use by queued decodes)
  const size_t tab_off = 256;
  const size_t bytes = tab_off + hd::table_bytes(K, alphabet);
  char* buf = nullptr;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  FieldDesc d{};
  d.lengths = lengths;
  d.alphabet = alphabet;
  d.table = reinterpret_cast<const hd::TableHeader*>(buf + tab_off);
  d.err = reinterpret_cast<uint32_t*>(buf);
  hd::PrepParams pp{};
  pp.f0 = d;
  pp.nfields = 1;
  pp.slices = kTableSlices;
  pp.table_blocks = kTableSlices;
  pp.K = K;
  int rc = HD_OK;
  uint32_t status = 1;
  const size_t n = size_t{1} << K;
  if (cudaMemsetAsync(buf, 0, tab_off, st) != cudaSuccess ||
      hd::launch_prepare(pp, st) != cudaSuccess ||
      cudaMemcpyAsync(&status, buf + tab_off, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (lut16 && cudaMemcpyAsync(lut16, buf + tab_off + hd::table_lut16_off(K, alphabet), 2 * n,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      (len8 && cudaMemcpyAsync(len8, buf + tab_off + hd::table_len8_off(K, alphabet), n,
                               cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      (run8 && cudaMemcpyAsync(run8, buf + tab_off + hd::table_run8_off(K, alphabet), n,
                               cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      (pair && cudaMemcpyAsync(pair, buf + tab_off + hd::table_pair_off(K, alphabet), 4 * n,
                               cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    rc = HD_ERR_CUDA;
  }
  cudaFree(buf);
  if (rc == HD_OK && status != 0) rc = HD_ERR_CORRUPT;
  return rc;
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
  if (c->recon_active) {
    uint32_t r = 0;
    if (cudaMemcpy(&r, c->rws, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    all |= r;
  }
  return map_err_bits(all);
}

int hd_decode_batch(hd_ctx* c, const hd_field* fs, uint32_t nf, uint16_t* const* d_outs,
                    void* stream) {
  if (!c || (nf && (!fs || !d_outs))) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return decode_batch_locked(c, fs, nf, d_outs, stream);
}

int hd_autotune(hd_ctx* c, const hd_field* fs, uint32_t nf, uint16_t* const* d_outs,
                void* stream, hd_config* best) {
  if (!c || !nf || !fs || !d_outs) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  for (uint32_t i = 0; i < nf; ++i) {
    const int rc = check_field(&fs[i], true, d_outs[i]);
    if (rc != HD_OK && rc != HD_PENDING) return rc;
  }
  BatchPlan plan;
  int rc = plan_batch(c, fs, nf, d_outs, plan);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hd_config saved = c->cfg;
  const bool saved_profile = c->profile;
  c->profile = false;
  cudaEvent_t t0 = c->tune_ev[0], t1 = c->tune_ev[1];
  bool first_group = true;
  for (int grp = 0; grp < 2 && rc == HD_OK; ++grp) {
    const bool ss = grp == 1;
    const std::vector<uint32_t>& idx = ss ? plan.sync_i : plan.gap_i;
    if (idx.empty()) continue;
    uint32_t maxS = 0;
    uint64_t bits = 0, syms = 0;
    for (uint32_t i : idx) {
      maxS = std::max(maxS, fs[i].subseq_bits);
      bits += fs[i].nbits;
      syms += fs[i].n;
    }
    const uint32_t S_list[4] = {64, 128, 256, 512};
    const uint32_t B_list[3] = {128, 256, 512};
    const uint32_t K_list[4] = {11, 12, 13, 14};
    double best_ms = 1e30;
    hd_config best_cfg{};
    // a single gap-array field: the one-pass decoder's shapes too (direct
    // launches, as hd_decode runs them)
    if (!ss && idx.size() == 1) {
      const uint32_t i = idx[0];
      for (uint32_t S : S_list) {
        if (S < 128 || S % maxS) continue;
        for (uint32_t B : {256u, 512u, 768u}) {
          for (uint32_t K : {12u, 13u, 14u}) {
            c->cfg = hd_config{S, B, 0, K, 0, 2};
            const hd::LaunchShape sh = group_shape(c, fs, idx, true);
            double ms = 1e30;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {
              std::vector<FieldDesc> dd(1);
              fill_desc(dd[0], &fs[i], sh, d_outs[i]);
              cudaEventRecord(t0, st);
              const int r = queue_decode(c, dd, sh, false, false, st);
              cudaEventRecord(t1, st);
              std::vector<uint32_t> bits_v;
              if (r || read_errors(c, stream, bits_v) != HD_OK) {
                ok = false;
                break;
              }
              for (uint32_t b : bits_v) ok &= b == 0;
              float t = 0;
              cudaEventElapsedTime(&t, t0, t1);
              if (rep) ms = std::min(ms, static_cast<double>(t));
            }
            if (ok && ms < best_ms) {
              best_ms = ms;
              best_cfg = hd_config{S, B, 0, K, 0, 2};
            }
          }
        }
      }
    }
    for (uint32_t S : S_list) {
      if (ss ? (S > 256) : (S < 128 || S % maxS)) continue;
      for (uint32_t B : B_list) {
        for (uint32_t K : K_list) {
          c->cfg = hd_config{S, B, 0, K, 0, 1};
          std::vector<FieldDesc> d;
          const hd::LaunchShape sh = group_shape(c, fs, idx, !ss);
          for (uint32_t i : idx) {
            FieldDesc x;
            fill_desc(x, &fs[i], sh, d_outs[i]);
            d.push_back(x);
          }
          double ms = 1e30;
          bool ok = true;
          for (int rep = 0; rep < 4 && ok; ++rep) {
            std::vector<FieldDesc> dd = d;
            cudaEventRecord(t0, st);
            const int r = queue_decode_graph(c, dd, sh, ss, st);
            cudaEventRecord(t1, st);
            if (r) {
              ok = false;
              break;
            }
            std::vector<uint32_t> bits_v;
            if (read_errors(c, stream, bits_v) != HD_OK) {
              ok = false;
              break;
            }
            for (uint32_t b : bits_v) ok &= b == 0;
            float t = 0;
            cudaEventElapsedTime(&t, t0, t1);
            if (rep) ms = std::min(ms, static_cast<double>(t));
          }
          if (ok && ms < best_ms) {
            best_ms = ms;
            best_cfg = hd_config{S, B, 0, K, 0, 1};
          }
        }
      }
    }
    if (best_ms >= 1e30) {
      rc = HD_ERR_CORRUPT;  // no candidate decoded the batch cleanly
      break;
    }
    c->tuned[tune_key(!ss, maxS, bits, syms)] = best_cfg;
    if (first_group && best) *best = best_cfg;
    first_group = false;
  }
  c->cfg = saved;
  c->profile = saved_profile;
  drop_graphs(c);  // keep only what later batches use (recaptured on demand)
  c->err_count = 0;
  c->recon_active = false;
  c->err_map.clear();
  return rc;
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
  if (f->gap && f->nbits && f->n) {
    bool used = false;
    rc = decode_host_pipelined(c, f, host_out, st, &used);
    if (rc) return rc;
    if (used) {
      std::vector<uint32_t> bits;
      rc = read_errors(c, stream, bits);
      if (rc) return rc;
      uint32_t all = 0;
      for (uint32_t b : bits) all |= b;
      return map_err_bits(all);
    }
  }
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

int hd_histogram_device(hd_ctx* c, const uint16_t* d_codes, uint64_t n, uint32_t alphabet,
                        uint64_t* freq_out, void* stream) {
  if (!c || !freq_out || (n && !d_codes)) return HD_ERR_ARG;
  if (alphabet < 1 || alphabet > 65536) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ensure_ws(c, 256 + 8ull * alphabet);
  if (rc) return rc;
  char* ws = c->ws;
  uint32_t err = 0;
  auto* hist = reinterpret_cast<unsigned long long*>(ws + 256);
  if (cudaMemsetAsync(ws, 0, 256 + 8ull * alphabet, st) != cudaSuccess ||
      hd::launch_histogram(d_codes, n, alphabet, hist, reinterpret_cast<uint32_t*>(ws),
                           c->num_sms, st) != cudaSuccess ||
      cudaMemcpyAsync(freq_out, hist, 8ull * alphabet, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(&err, ws, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  c->launches += n ? 1 : 0;
  c->err_count = 0;
  c->recon_active = false;
  return err ? HD_ERR_SYMBOL : HD_OK;
}

int hd_encode_device(hd_ctx* c, const uint16_t* d_codes, uint64_t n, const uint8_t* lengths,
                     uint32_t alphabet, uint32_t subseq_bits, uint32_t* d_words,
                     uint64_t words_cap, uint8_t* d_gap, uint64_t gap_cap, hd_stream_info* info,
                     void* stream) {
  if (!c || !info || !lengths || (n && !d_codes)) return HD_ERR_ARG;
  if (alphabet < 1 || alphabet > 65536) return HD_ERR_ARG;
  if (subseq_bits != 64 && subseq_bits != 128 && subseq_bits != 256) return HD_ERR_ARG;
  if (d_codes && (reinterpret_cast<uintptr_t>(d_codes) & 1u)) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  std::vector<uint32_t> cw(alphabet);
  int rc = hd::canonical_codewords(lengths, alphabet, cw.data());
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t tiles = hd::encode_tiles(n);
  // workspace: error word | lengths | codewords | tile bits | tile offsets
  const size_t err_off = 0;
  const size_t len_off = 256;
  const size_t cw_off = align_up(len_off + alphabet, 256);
  const size_t tb_off = align_up(cw_off + 4ull * alphabet, 256);
  const size_t to_off = align_up(tb_off + 4ull * tiles, 256);
  rc = ensure_ws(c, to_off + 8ull * (tiles + 1));
  if (rc) return rc;
  char* ws = c->ws;
  c->err_count = 0;  // hd_status does not report encodes
  c->recon_active = false;
  hd::EncodeParams e{};
  e.codes = d_codes;
  e.n = n;
  e.lengths = reinterpret_cast<const uint8_t*>(ws + len_off);
  e.codewords = reinterpret_cast<const uint32_t*>(ws + cw_off);
  e.alphabet = alphabet;
  e.subseq_bits = subseq_bits;
  e.tiles = tiles;
  e.tile_bits = reinterpret_cast<uint32_t*>(ws + tb_off);
  e.tile_off = reinterpret_cast<uint64_t*>(ws + to_off);
  e.err = reinterpret_cast<uint32_t*>(ws + err_off);
  uint64_t nbits = 0;
  uint32_t err = 0;
  if (cudaMemsetAsync(ws + err_off, 0, 16, st) != cudaSuccess ||
      cudaMemcpyAsync(ws + len_off, lengths, alphabet, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ws + cw_off, cw.data(), 4ull * alphabet, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      hd::launch_encode_count(e, c->num_sms, st) != cudaSuccess)
    return HD_ERR_CUDA;
  c->launches += tiles ? 2 : 0;
  if ((tiles && cudaMemcpyAsync(&nbits, ws + to_off + 8 * tiles, 8, cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess) ||
      cudaMemcpyAsync(&err, ws + err_off, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  if (err) return HD_ERR_SYMBOL;
  const uint32_t S = subseq_bits;
  info->nbits = nbits;
  info->nsub = (nbits + S - 1) / S;
  info->nwords = hd::stream_words(nbits, S);
  if (!d_words || words_cap < info->nwords) return HD_ERR_CAPACITY;
  if (d_gap && gap_cap < info->nsub) return HD_ERR_CAPACITY;
  if (reinterpret_cast<uintptr_t>(d_words) & 3u) return HD_ERR_ARG;
  e.words = d_words;
  e.gap = d_gap;
  e.nsub = info->nsub;
  if (cudaMemsetAsync(d_words, 0, 4ull * info->nwords, st) != cudaSuccess ||
      hd::launch_encode_write(e, c->num_sms, st) != cudaSuccess)
    return HD_ERR_CUDA;
  c->launches += tiles ? 1 : 0;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_CUDA;
  }
  return HD_OK;
}

// ---- Lorenzo reconstruction -------------------------------------------------

static constexpr uint64_t kReconMaxRow = 49152;          // 2D/3D row limit (band shared memory)
static constexpr uint64_t kReconGroupBytes = 32ull << 20;  // int32 intermediate per slice group

static int ensure_rws(hd_ctx* c, size_t need) {
  if (need <= c->rws_cap) return HD_OK;
  if (c->rws) {
    cudaDeviceSynchronize();
    cudaFree(c->rws);
    c->rws = nullptr;
    c->rws_cap = 0;
  }
  const size_t cap = align_up(std::max<size_t>(need, 1 << 20), 1 << 20);
  if (cudaMalloc(&c->rws, cap) != cudaSuccess) {
    cudaGetLastError();
    return HD_ERR_NOMEM;
  }
  c->rws_cap = cap;
  return HD_OK;
}

// Argument checks shared by the reconstruction entry points; n receives the
// grid size.
static int check_lorenzo(const hd_lorenzo* L, uint64_t* n) {
  if (!L || L->ndim < 1 || L->ndim > 3) return HD_ERR_ARG;
  if (L->radius < 1 || L->radius > 32768) return HD_ERR_ARG;
  if (!(L->eb >= 0.0) || !std::isfinite(L->eb)) return HD_ERR_ARG;
  if (!std::isfinite(static_cast<float>(2.0 * L->eb))) return HD_ERR_ARG;
  uint64_t m = 1;
  for (uint32_t k = 0; k < L->ndim; ++k) {
    const uint64_t e = L->dims[k];
    if (e && m > (1ull << 48) / e) return HD_ERR_ARG;
    m *= e;
  }
  if (L->n_out > m || (L->n_out && (!L->out_idx || !L->out_val))) return HD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(L->out_idx) & 7u) || (reinterpret_cast<uintptr_t>(L->out_val) & 3u))
    return HD_ERR_ARG;
  *n = m;
  return HD_OK;
}

// Decode + 1D reconstruction of one gap-array field in the decoder's kernels.
static int decompress_fused_1d(hd_ctx* c, const hd_field* f, const hd_lorenzo* L, float* d_out,
                               void* stream) {
  c->err_count = 0;
  c->recon_active = false;
  c->host_status = HD_ERR_ARG;
  uint64_t n = 0;
  int rc = check_lorenzo(L, &n);
  if (rc) return rc;
  if (n && (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 15u))) return HD_ERR_ARG;
  rc = check_field(f, true, d_out);
  if (rc == HD_PENDING) {
    c->host_status = HD_OK;
    return HD_OK;
  }
  if (rc) {
    c->host_status = rc;
    return rc;
  }
  if (f->nbits == 0 || f->n == 0) {
    c->host_status = HD_ERR_CORRUPT;
    return HD_OK;
  }
  hd::LaunchShape s = field_shape(c, f, true);
  if (s.S % f->subseq_bits) return HD_ERR_ARG;
  if (ensure_rws(c, 256) != HD_OK) {
    c->host_status = HD_ERR_NOMEM;
    return HD_ERR_NOMEM;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(c->rws, 0, 4, st) != cudaSuccess) {
    cudaGetLastError();
    c->host_status = HD_ERR_CUDA;
    return HD_ERR_CUDA;
  }
  std::vector<FieldDesc> descs(1);
  fill_desc(descs[0], f, s, nullptr);
  ValueArgs va{d_out, static_cast<int32_t>(L->radius), static_cast<float>(2.0 * L->eb),
               L->out_idx, L->out_val, L->n_out, reinterpret_cast<uint32_t*>(c->rws)};
  rc = queue_decode(c, descs, s, false, false, st, &va);
  c->host_status = rc;
  if (rc == HD_OK) c->recon_active = true;
  return rc;
}

static int reconstruct_locked(hd_ctx* c, const uint16_t* d_codes, const hd_lorenzo* L,
                              float* d_out, void* stream) {
  c->err_count = 0;
  c->recon_active = false;
  c->host_status = HD_ERR_ARG;
  if (!L || L->ndim < 1 || L->ndim > 3) return HD_ERR_ARG;
  if (L->radius < 1 || L->radius > 32768) return HD_ERR_ARG;
  if (!(L->eb >= 0.0) || !std::isfinite(L->eb)) return HD_ERR_ARG;
  const float ebx2 = static_cast<float>(2.0 * L->eb);
  if (!std::isfinite(ebx2)) return HD_ERR_ARG;
  uint64_t ext[3] = {1, 1, 1};
  uint64_t n = 1;
  for (uint32_t k = 0; k < L->ndim; ++k) {
    ext[k] = L->dims[k];
    if (ext[k] && n > (1ull << 48) / ext[k]) return HD_ERR_ARG;
    n *= ext[k];
  }
  if (L->n_out > n || (L->n_out && (!L->out_idx || !L->out_val))) return HD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(L->out_idx) & 7u) || (reinterpret_cast<uintptr_t>(L->out_val) & 3u))
    return HD_ERR_ARG;
  if (n && (!d_codes || !d_out)) return HD_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_codes) & 15u) || (reinterpret_cast<uintptr_t>(d_out) & 15u))
    return HD_ERR_ARG;
  const bool one_d = L->ndim == 1;
  if (!one_d && ext[0] > kReconMaxRow) return HD_ERR_ARG;
  if (one_d && hd::lorenzo_tiles_1d(n) > 0x7fffffffull) return HD_ERR_ARG;
  if (!one_d && L->band_rows > 64) return HD_ERR_ARG;
  if (!n) {
    c->host_status = HD_OK;
    return HD_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  hd::LorenzoParams P{};
  P.codes = d_codes;
  P.out = d_out;
  P.n = n;
  P.radius = static_cast<int32_t>(L->radius);
  P.ebx2 = ebx2;
  P.out_idx = L->out_idx;
  P.out_val = L->out_val;
  P.n_out = L->n_out;
  size_t need = 256;
  uint64_t zc = 1;
  // 3D grids with many slices and rows up to 1024 codes: one block per
  // slice, then the z kernel (no band carries); a launch shape given for the
  // band path selects that instead
  const bool slice_path = L->ndim == 3 && !L->chunk_slices && !L->band_rows &&
                          hd::lorenzo_slice_path(ext[0], ext[2], c->num_sms);
  if (one_d) {
    P.nx = n;
    P.ny = P.nz = 1;
    need += 4ull * hd::lorenzo_tiles_1d(n);
  } else if (slice_path) {
    P.nx = ext[0];
    P.ny = ext[1];
    P.nz = ext[2];
  } else {
    P.nx = ext[0];
    P.ny = ext[1];
    P.nz = L->ndim == 3 ? ext[2] : 1;
    P.yb = L->band_rows ? L->band_rows : hd::lorenzo_rows_per_band(P.nx);
    P.nb = (P.ny + P.yb - 1) / P.yb;
    const uint64_t plane_bytes = 4ull * P.ny * P.nx;
    zc = L->chunk_slices ? L->chunk_slices
                         : std::max<uint64_t>(1, kReconGroupBytes / plane_bytes);
    zc = std::min<uint64_t>(zc, P.nz);
    if (hd::lorenzo_band_smem(P.yb, P.nx) > static_cast<size_t>(c->max_smem)) return HD_ERR_ARG;
    if (zc * P.nb > 0x7fffffffull) zc = std::max<uint64_t>(1, 0x7fffffffull / P.nb);
    need = align_up(need, 256) + align_up(4ull * zc * P.nb * P.nx, 256) + plane_bytes;
  }
  c->host_status = HD_OK;
  if (ensure_rws(c, need) != HD_OK) {
    c->host_status = HD_ERR_NOMEM;
    return HD_ERR_NOMEM;
  }
  P.err = reinterpret_cast<uint32_t*>(c->rws);
  P.tile_prefix = reinterpret_cast<int32_t*>(c->rws + 256);
  P.band = reinterpret_cast<int32_t*>(c->rws + 256);
  P.plane = reinterpret_cast<int32_t*>(c->rws + 256 + align_up(4ull * zc * P.nb * P.nx, 256));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->profile) {
    e0 = next_event(c);
    e1 = next_event(c);
  }
  cudaError_t e = cudaMemsetAsync(c->rws, 0, 4, st);
  if (e == cudaSuccess && c->profile) e = cudaEventRecord(e0, st);
  uint64_t launches = 0;
  if (one_d) {
    if (e == cudaSuccess) e = hd::launch_lorenzo_1d(P, c->num_sms, st);
    launches = 3;
  } else if (slice_path) {
    P.z_lo = 0;
    P.z_hi = P.nz;
    if (e == cudaSuccess) e = hd::launch_lorenzo_whole_slices(P, c->num_sms, st);
    launches = 2;
  } else {
    for (uint64_t z = 0; z < P.nz && e == cudaSuccess; z += zc) {
      P.z_lo = z;
      P.z_hi = std::min(P.nz, z + zc);
      e = hd::launch_lorenzo_slices(P, c->num_sms, st);
      launches += 3;
    }
  }
  if (e == cudaSuccess && c->profile) {
    e = cudaEventRecord(e1, st);
    c->spans.emplace_back(e0, e1);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->host_status = HD_ERR_CUDA;
    return HD_ERR_CUDA;
  }
  c->launches += launches;
  c->recon_active = true;
  return HD_OK;
}

int hd_reconstruct_device(hd_ctx* c, const uint16_t* d_codes, const hd_lorenzo* L, float* d_out,
                          void* stream) {
  if (!c) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  return reconstruct_locked(c, d_codes, L, d_out, stream);
}

int hd_decompress_device(hd_ctx* c, const hd_field* f, const hd_lorenzo* L, float* d_out,
                         void* stream) {
  if (!c || !f || !L) return HD_ERR_ARG;
  uint64_t n = 1;
  for (uint32_t k = 0; k < L->ndim && k < 3; ++k) n *= L->dims[k];
  if (L->ndim < 1 || L->ndim > 3 || f->n != n) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  if (L->ndim == 1 && f->gap && !L->separate && !c->cfg.cr_classes)
    return decompress_fused_1d(c, f, L, d_out, stream);
  const size_t bytes = align_up(2 * n + 16, 256);
  if (bytes > c->dcodes_cap) {
    if (c->dcodes) {
      cudaDeviceSynchronize();
      cudaFree(c->dcodes);
      c->dcodes = nullptr;
      c->dcodes_cap = 0;
    }
    if (cudaMalloc(&c->dcodes, bytes) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_NOMEM;
    }
    c->dcodes_cap = bytes;
  }
  int rc = decode_impl(c, f, c->dcodes, nullptr, stream);
  if (rc) return rc;
  if (c->host_status != HD_OK) return HD_OK;  // hd_status reports it; nothing to reconstruct
  const uint32_t err_words = c->err_count;
  const size_t err_off = c->err_off;
  rc = reconstruct_locked(c, c->dcodes, L, d_out, stream);
  // hd_status reports the decode's error words and the reconstruction's
  c->err_count = err_words;
  c->err_off = err_off;
  return rc;
}

int hd_set_wait_limit(hd_ctx* c, uint64_t cycles) {
  if (!c) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  c->wait_limit = cycles;
  return HD_OK;
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
  for (const auto& pr : c->spans) {
    if (cudaEventSynchronize(pr.second) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    float t = 0;
    if (cudaEventElapsedTime(&t, pr.first, pr.second) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    total += t;
    ++n;
  }
  c->spans.clear();
  if (c->phase_recs.empty()) c->events_used = 0;
  *ms = total;
  *launches = n;
  return HD_OK;
}

int hd_phase_times(hd_ctx* c, double* ms, uint64_t* decodes) {
  if (!c || !ms || !decodes) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  DeviceGuard g(c->device);
  for (int k = 0; k < 4; ++k) ms[k] = 0;
  uint64_t n = 0;
  for (const auto& r : c->phase_recs) {
    const cudaEvent_t a = std::get<1>(r), b = std::get<2>(r);
    float t = 0;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess) {
      cudaGetLastError();
      return HD_ERR_CUDA;
    }
    ms[std::get<0>(r)] += t;
    n += std::get<0>(r) == kPhWrite ? 1 : 0;
  }
  c->phase_recs.clear();
  if (c->spans.empty()) c->events_used = 0;
  *decodes = n;
  return HD_OK;
}

uint64_t hd_launch_count(hd_ctx* c) { return c ? c->launches : 0; }

// GPU name without spaces (the key of a saved autotuner entry).
static std::string gpu_key(int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string k = prop.name;
  for (char& ch : k)
    if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
  return k;
}

int hd_autotune_save(hd_ctx* c, const char* path) {
  if (!c || !path) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  const std::string gpu = gpu_key(c->device);
  FILE* f = std::fopen(path, "w");
  if (!f) return HD_ERR_ARG;
  std::fprintf(f, "hd-autotune 1\n");
  for (const auto& kv : c->tuned) {
    const hd_config& x = kv.second;
    std::fprintf(f, "%s %u %u %u %u %u %u %u %u %u %u\n", gpu.c_str(),
                 std::get<0>(kv.first) ? 1u : 0u, std::get<1>(kv.first), std::get<2>(kv.first),
                 std::get<3>(kv.first), x.subseq_bits, x.threads, x.window, x.lut_bits,
                 x.cr_classes, x.decoder);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? HD_OK : HD_ERR_ARG;
}

int hd_autotune_load(hd_ctx* c, const char* path, uint32_t* loaded) {
  if (!c || !path || !loaded) return HD_ERR_ARG;
  *loaded = 0;
  std::lock_guard<std::mutex> lk(c->mu);
  const std::string gpu = gpu_key(c->device);
  FILE* f = std::fopen(path, "r");
  if (!f) return HD_ERR_ARG;
  char head[32] = {0};
  int rc = HD_OK;
  if (std::fscanf(f, "%31s", head) != 1 || std::strcmp(head, "hd-autotune") != 0) rc = HD_ERR_ARG;
  unsigned ver = 0;
  if (rc == HD_OK && (std::fscanf(f, "%u", &ver) != 1 || ver != 1)) rc = HD_ERR_ARG;
  std::map<TuneKey, hd_config> got;
  while (rc == HD_OK) {
    char name[256];
    unsigned ss, qb, lg, ms, S, B, W, K, cr, dec;
    const int k = std::fscanf(f, "%255s %u %u %u %u %u %u %u %u %u %u", name, &ss, &qb, &lg, &ms,
                              &S, &B, &W, &K, &cr, &dec);
    if (k == EOF) break;
    if (k != 11) {
      rc = HD_ERR_ARG;
      break;
    }
    // the same checks as hd_set_config: a shape the library would refuse is
    // no entry
    const hd_config x{S, B, W, K, cr, dec};
    const bool okS = (S == 64 || S == 128 || S == 256 || S == 512);
    const bool okB = B == 128 || B == 256 || B == 512 || ((B == 768 || B == 1024) && dec == 2);
    if (!okS || !okB || (K && (K < 8 || K > 15)) || dec > 2 || cr > 32 || ss > 1) {
      rc = HD_ERR_ARG;
      break;
    }
    if (gpu == name) got[TuneKey{ss != 0, qb, lg, ms}] = x;
  }
  std::fclose(f);
  if (rc) return rc;
  for (const auto& kv : got) c->tuned[kv.first] = kv.second;
  *loaded = static_cast<uint32_t>(got.size());
  return HD_OK;
}

int hd_graph_stats(hd_ctx* c, uint64_t* captures, uint32_t* cached) {
  if (!c || !captures || !cached) return HD_ERR_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  *captures = c->captures;
  *cached = static_cast<uint32_t>(c->graphs.size());
  return HD_OK;
}

}  // extern "C"
