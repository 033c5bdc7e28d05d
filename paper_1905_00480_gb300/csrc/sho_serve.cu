// sho_serve.cu -- continuous-batching request loop over device-resident systems (the sho_server_*
// part of include/sho.h).
//
// One scheduler thread owns `slots` execution slots (stream + handle/workspace + completion event).
// It repeatedly (1) retires slots whose completion event has fired, recording the request latency,
// and (2) starts queued requests whose system is idle and for which a free slot exists whose workspace,
// grown to the request's need, keeps resident systems + all slot workspaces within the memory budget:
// the earliest request of each system is a candidate, and the candidate with the smallest expected
// service time minus its waiting time goes first (shortest job first with aging).  Requests that arrive while others
// run are admitted as soon as a slot and memory free up; requests of different systems overlap on the
// device.  Nothing here waits on the device without a bound: completion is polled with
// cudaEventQuery, and host waits (sho_wait) take a timeout.  A finished request's status includes the
// device status word of its slot's handle (a kernel's expired bounded wait, an out-of-range input).
// Each request is an NVTX range ("sho project/expand sys=<id>") from its start to its retirement.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sho_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

// Service-rate estimate of the admission order: algorithmic bytes per second of one request on the GPU.
constexpr double kServeBytesPerSecond = 500e9;

struct SysRec {
  sho_grid grid;
  int nbands = 0, natoms = 0, numax = 0, cube = 0;
  sho_dtype psi_dt = SHO_F32, coeff_dt = SHO_F32;
  std::vector<double> pos, sigma;
  void* psi = nullptr;
  void* coeff = nullptr;
  size_t psi_bytes = 0, coeff_bytes = 0;
  bool busy = false;
  bool held = false;  // fault injection: a running request of this system is not retired
  int pending = 0;    // queued + running requests
  double bytes_prj = 0.0, bytes_add = 0.0;
};

struct Req {
  int sys = -1;
  sho_op op = SHO_OP_PROJECT;
  sho_prec prec = SHO_P_FP32;
  size_t need = 0;
  double t_submit = 0.0, t_done = 0.0;
  int status = SHO_OK;
  bool done = false;
};

struct Slot {
  cudaStream_t stream = nullptr;
  sho_handle* h = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  uint64_t ticket = 0;
  nvtxRangeId_t range = 0;
};

// Distinct grid points covered by the cubes (algorithmic psi traffic of one request).
double union_points(const sho_grid& g, const std::vector<double>& pos, int natoms, int cube) {
  const size_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
  std::vector<uint8_t> mask(nx * ny * nz, 0);
  for (int a = 0; a < natoms; a++) {
    int o[3];
    for (int d = 0; d < 3; d++) o[d] = (int)std::floor(pos[3 * a + d] / g.h) - cube / 2 + 1;
    for (int iz = 0; iz < cube; iz++) {
      int jz = o[2] + iz;
      if (g.periodic) jz = ((jz % (int)nz) + (int)nz) % (int)nz;
      else if (jz < 0 || jz >= (int)nz) continue;
      for (int iy = 0; iy < cube; iy++) {
        int jy = o[1] + iy;
        if (g.periodic) jy = ((jy % (int)ny) + (int)ny) % (int)ny;
        else if (jy < 0 || jy >= (int)ny) continue;
        uint8_t* row = &mask[((size_t)jz * ny + jy) * nx];
        for (int ix = 0; ix < cube; ix++) {
          int jx = o[0] + ix;
          if (g.periodic) jx = ((jx % (int)nx) + (int)nx) % (int)nx;
          else if (jx < 0 || jx >= (int)nx) continue;
          row[jx] = 1;
        }
      }
    }
  }
  size_t c = 0;
  for (uint8_t m : mask) c += m;
  return (double)c;
}

}  // namespace

struct sho_server {
  int device = 0;
  size_t budget = 0;
  std::vector<Slot> slots;
  std::map<int, SysRec> systems;
  int next_sys = 1;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> queue;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
  bool stop = false;
  // accounting
  size_t resident = 0, peak = 0;
  int inflight = 0, max_inflight = 0;
  uint64_t submitted = 0, completed = 0, failed = 0;
  std::vector<double> lat_ms;
  double t_first = -1.0, t_last = 0.0, bytes_done = 0.0;

  size_t workspaces() const {
    size_t s = 0;
    for (const Slot& sl : slots) s += sho::handle_workspace(sl.h);
    return s;
  }
};

namespace {

void note_peak(sho_server* s) { s->peak = std::max(s->peak, s->resident + s->workspaces()); }

// Pick a free slot for a request needing `need` workspace bytes, or -1.
int pick_slot(sho_server* s, size_t need) {
  const size_t total_ws = s->workspaces();
  int best = -1;
  size_t best_growth = (size_t)-1;
  for (size_t k = 0; k < s->slots.size(); k++) {
    const Slot& sl = s->slots[k];
    if (sl.busy) continue;
    const size_t ws = sho::handle_workspace(sl.h);
    const size_t grown = std::max(ws, need);
    if (s->resident + (total_ws - ws) + grown > s->budget) continue;
    const size_t growth = grown - ws;
    if (growth < best_growth) {
      best_growth = growth;
      best = (int)k;
    }
  }
  return best;
}

void finish(sho_server* s, Slot& sl, int status) {
  Req& r = s->reqs[sl.ticket];
  r.status = status;
  r.done = true;
  r.t_done = now_s();
  SysRec& sys = s->systems[r.sys];
  sys.busy = false;
  sys.pending--;
  sl.busy = false;
  if (sl.range) nvtxRangeEnd(sl.range);
  sl.range = 0;
  s->inflight--;
  s->completed++;
  if (status != SHO_OK) s->failed++;
  s->lat_ms.push_back((r.t_done - r.t_submit) * 1e3);
  s->t_last = r.t_done;
  if (status == SHO_OK) s->bytes_done += (r.op == SHO_OP_PROJECT) ? sys.bytes_prj : sys.bytes_add;
}

void start(sho_server* s, int k, uint64_t ticket) {
  Slot& sl = s->slots[(size_t)k];
  Req& r = s->reqs[ticket];
  SysRec& sys = s->systems[r.sys];
  sl.busy = true;
  sl.ticket = ticket;
  sys.busy = true;
  s->inflight++;
  s->max_inflight = std::max(s->max_inflight, s->inflight);
  if (s->t_first < 0.0) s->t_first = now_s();
  char name[64];
  std::snprintf(name, sizeof(name), "sho %s sys=%d", r.op == SHO_OP_PROJECT ? "project" : "expand", r.sys);
  sl.range = nvtxRangeStartA(name);
  int st = sho::handle_reserve(sl.h, r.need);
  note_peak(s);
  if (st == SHO_OK) {
    if (r.op == SHO_OP_PROJECT)
      st = sho_project(sl.h, &sys.grid, sys.psi, sys.psi_dt, sys.nbands, sys.natoms, sys.pos.data(), sys.sigma.data(),
                       sys.numax, sys.cube, r.prec, sys.coeff, sys.coeff_dt, sl.stream);
    else
      st = sho_add(sl.h, &sys.grid, sys.coeff, sys.coeff_dt, sys.nbands, sys.natoms, sys.pos.data(), sys.sigma.data(),
                   sys.numax, sys.cube, r.prec, sys.psi, sys.psi_dt, sl.stream);
  }
  if (st == SHO_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = SHO_ERR_CUDA;
  if (st != SHO_OK) finish(s, sl, st);
}

void scheduler(sho_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progress = false;
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      if (s->systems[s->reqs[sl.ticket].sys].held) continue;  // fault injection: a stuck request
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      // the request's kernels are done: fold in what they reported through the handle's status word
      int st = q == cudaSuccess ? sho::handle_take_status(sl.h) : SHO_ERR_CUDA;
      if (q != cudaSuccess) cudaGetLastError();
      finish(s, sl, st);
      progress = true;
    }
    if (!s->stop) {
      // Admission order: among the earliest queued request of every idle system (a system's requests
      // run in submission order), start the one with the smallest expected service time minus the time
      // it has waited -- shortest job first, aged so that a large request waits at most about its own
      // service time longer than small ones -- while a slot and memory allow.
      for (;;) {
        const double tnow = now_s();
        auto best = s->queue.end();
        double best_score = 0.0;
        int best_slot = -1;
        std::vector<int> seen;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
          const Req& r = s->reqs[*it];
          if (std::find(seen.begin(), seen.end(), r.sys) != seen.end()) continue;
          seen.push_back(r.sys);
          const SysRec& sys = s->systems[r.sys];
          if (sys.busy) continue;
          const double est = (r.op == SHO_OP_PROJECT ? sys.bytes_prj : sys.bytes_add) / kServeBytesPerSecond;
          const double score = est - (tnow - r.t_submit);
          if (best != s->queue.end() && score >= best_score) continue;
          const int k = pick_slot(s, r.need);
          if (k < 0) continue;
          best = it;
          best_score = score;
          best_slot = k;
        }
        if (best == s->queue.end()) break;
        const uint64_t t = *best;
        s->queue.erase(best);
        start(s, best_slot, t);
        progress = true;
      }
    }
    if (progress) s->cv_done.notify_all();
    if (s->stop && s->inflight == 0) break;
    if (!progress) s->cv_work.wait_for(lk, std::chrono::microseconds(20));
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int sho_server_create(sho_server** out, int device, size_t budget_bytes, int slots) {
  if (!out || slots <= 0 || slots > 64 || budget_bytes == 0) return SHO_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return SHO_ERR_CUDA;
  }
  if (device < 0 || device >= count) return SHO_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return SHO_ERR_CUDA;
  sho_server* s = new sho_server();
  s->device = device;
  s->budget = budget_bytes;
  s->slots.resize((size_t)slots);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        sho_create(&sl.h, device) != SHO_OK) {
      for (Slot& t : s->slots) {
        if (t.h) sho_destroy(t.h);
        if (t.done) cudaEventDestroy(t.done);
        if (t.stream) cudaStreamDestroy(t.stream);
      }
      delete s;
      return SHO_ERR_CUDA;
    }
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return SHO_OK;
}

int sho_server_destroy(sho_server* s) {
  if (!s) return SHO_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& kv : s->systems) kv.second.held = false;  // held requests retire once their work is done
    for (uint64_t t : s->queue) {
      Req& r = s->reqs[t];
      r.status = SHO_ERR_STATE;
      r.done = true;
      s->systems[r.sys].pending--;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->th.join();
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    sho_destroy(sl.h);
    cudaEventDestroy(sl.done);
    cudaStreamDestroy(sl.stream);
  }
  for (auto& kv : s->systems) {
    cudaFree(kv.second.psi);
    cudaFree(kv.second.coeff);
  }
  delete s;
  return SHO_OK;
}

int sho_system_register(sho_server* s, const sho_grid* grid, int nbands, int natoms, const double* pos,
                        const double* sigma, int numax, int cube, sho_dtype psi_dtype, const void* psi,
                        int* system_id) {
  if (!s || !grid || !system_id || !psi || nbands <= 0 || natoms < 0) return SHO_ERR_ARG;
  if (natoms > 0 && (!pos || !sigma)) return SHO_ERR_ARG;
  if (psi_dtype != SHO_F64 && psi_dtype != SHO_F32 && psi_dtype != SHO_BF16) return SHO_ERR_DTYPE;
  if (numax < 0 || numax > SHO_MAX_NUMAX) return SHO_ERR_NUMAX;
  if (cube < 8 || cube > sho::kMaxCube || cube % 8) return SHO_ERR_CUBE;
  for (int d = 0; d < 3; d++)
    if (grid->n[d] <= 0 || (grid->periodic && cube > grid->n[d])) return SHO_ERR_CUBE;
  SysRec r;
  r.grid = *grid;
  r.nbands = nbands;
  r.natoms = natoms;
  r.numax = numax;
  r.cube = cube;
  r.psi_dt = psi_dtype;
  r.coeff_dt = psi_dtype == SHO_F64 ? SHO_F64 : SHO_F32;
  r.pos.assign(pos, pos + 3 * (size_t)natoms);
  r.sigma.assign(sigma, sigma + (size_t)natoms);
  const size_t es = psi_dtype == SHO_F64 ? 8 : (psi_dtype == SHO_F32 ? 4 : 2);
  const size_t cs = r.coeff_dt == SHO_F64 ? 8 : 4;
  r.psi_bytes = (size_t)grid->n[0] * grid->n[1] * grid->n[2] * (size_t)nbands * es;
  r.coeff_bytes = (size_t)natoms * (size_t)sho::nstates(numax) * (size_t)nbands * cs;
  const double U = union_points(*grid, r.pos, natoms, cube);
  r.bytes_prj = U * nbands * (double)es + (double)r.coeff_bytes;
  r.bytes_add = 2.0 * U * nbands * (double)es + (double)r.coeff_bytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->resident + s->workspaces() + r.psi_bytes + r.coeff_bytes > s->budget) return SHO_ERR_CAPACITY;
  cudaSetDevice(s->device);
  if (cudaMalloc(&r.psi, r.psi_bytes) != cudaSuccess) {
    cudaGetLastError();
    return SHO_ERR_OOM;
  }
  if (cudaMalloc(&r.coeff, std::max<size_t>(r.coeff_bytes, 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(r.psi);
    return SHO_ERR_OOM;
  }
  if (cudaMemcpy(r.psi, psi, r.psi_bytes, cudaMemcpyDefault) != cudaSuccess ||
      cudaMemset(r.coeff, 0, std::max<size_t>(r.coeff_bytes, 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(r.psi);
    cudaFree(r.coeff);
    return SHO_ERR_CUDA;
  }
  s->resident += r.psi_bytes + r.coeff_bytes;
  note_peak(s);
  const int id = s->next_sys++;
  s->systems[id] = std::move(r);
  *system_id = id;
  return SHO_OK;
}

int sho_system_unregister(sho_server* s, int id) {
  if (!s) return SHO_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->systems.find(id);
  if (it == s->systems.end() || it->second.pending > 0) return SHO_ERR_STATE;
  cudaSetDevice(s->device);
  cudaFree(it->second.psi);
  cudaFree(it->second.coeff);
  s->resident -= it->second.psi_bytes + it->second.coeff_bytes;
  s->systems.erase(it);
  return SHO_OK;
}

static int system_copy(sho_server* s, int id, void* psi_out, void* coeff_out, const void* coeff_in) {
  if (!s) return SHO_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->systems.find(id);
  if (it == s->systems.end()) return SHO_ERR_STATE;
  // wait (bounded by the system's own requests) until nothing of this system is queued or running
  while (it->second.pending > 0) {
    s->cv_done.wait_for(lk, std::chrono::milliseconds(1));
    it = s->systems.find(id);
    if (it == s->systems.end()) return SHO_ERR_STATE;
  }
  SysRec& r = it->second;
  cudaSetDevice(s->device);
  if (psi_out && cudaMemcpy(psi_out, r.psi, r.psi_bytes, cudaMemcpyDefault) != cudaSuccess) return SHO_ERR_CUDA;
  if (coeff_out && r.coeff_bytes && cudaMemcpy(coeff_out, r.coeff, r.coeff_bytes, cudaMemcpyDefault) != cudaSuccess)
    return SHO_ERR_CUDA;
  if (coeff_in && r.coeff_bytes && cudaMemcpy(r.coeff, coeff_in, r.coeff_bytes, cudaMemcpyDefault) != cudaSuccess)
    return SHO_ERR_CUDA;
  return SHO_OK;
}

int sho_system_read(sho_server* s, int id, void* psi_out, void* coeff_out) {
  return system_copy(s, id, psi_out, coeff_out, nullptr);
}

int sho_system_write_coeff(sho_server* s, int id, const void* coeff_in) {
  if (!coeff_in) return SHO_ERR_ARG;
  return system_copy(s, id, nullptr, nullptr, coeff_in);
}

int sho_submit(sho_server* s, int id, sho_op op, sho_prec prec, uint64_t* ticket) {
  if (!s || !ticket || (op != SHO_OP_PROJECT && op != SHO_OP_EXPAND)) return SHO_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return SHO_ERR_STATE;
  auto it = s->systems.find(id);
  if (it == s->systems.end()) return SHO_ERR_STATE;
  SysRec& sys = it->second;
  const bool f64 = sys.psi_dt == SHO_F64;
  if (sho::is_f64_form(prec) != f64) return SHO_ERR_DTYPE;
  Req r;
  r.sys = id;
  r.op = op;
  r.prec = prec;
  r.need = sho::workspace_bytes(op, &sys.grid, sys.natoms, sys.numax, sys.cube, sys.nbands, sys.coeff_dt);
  if (s->resident + r.need > s->budget) return SHO_ERR_CAPACITY;
  r.t_submit = now_s();
  const uint64_t t = s->next_ticket++;
  s->reqs[t] = r;
  s->queue.push_back(t);
  sys.pending++;
  s->submitted++;
  *ticket = t;
  s->cv_work.notify_one();
  return SHO_OK;
}

int sho_wait_status(sho_server* s, uint64_t ticket, int timeout_ms, int* request_status, double* latency_ms) {
  if (!s || !request_status) return SHO_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SHO_ERR_STATE;
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  while (!s->reqs[ticket].done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->reqs[ticket].done)
      return SHO_ERR_TIMEOUT;
  }
  const Req& r = s->reqs[ticket];
  *request_status = r.status;
  if (latency_ms) latency_ms[0] = r.status == SHO_ERR_CANCELLED ? 0.0 : (r.t_done - r.t_submit) * 1e3;
  s->reqs.erase(ticket);
  return SHO_OK;
}

int sho_wait(sho_server* s, uint64_t ticket, int timeout_ms) {
  int st = SHO_OK;
  const int w = sho_wait_status(s, ticket, timeout_ms, &st, nullptr);
  return w != SHO_OK ? w : st;
}

int sho_cancel(sho_server* s, uint64_t ticket) {
  if (!s) return SHO_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || it->second.done) return SHO_ERR_STATE;
  auto q = std::find(s->queue.begin(), s->queue.end(), ticket);
  if (q == s->queue.end()) return SHO_ERR_STATE;  // already started: its GPU work is not interrupted
  s->queue.erase(q);
  Req& r = it->second;
  r.status = SHO_ERR_CANCELLED;
  r.done = true;
  r.t_done = now_s();
  s->systems[r.sys].pending--;
  s->cv_done.notify_all();
  return SHO_OK;
}

int sho_fault_server_pipeline(sho_server* s, long long cycles, int rows) {
  if (!s || cycles < 0) return SHO_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  for (Slot& sl : s->slots) {
    const int st = sho_fault_wait_limit(sl.h, cycles);
    if (st != SHO_OK) return st;
    sho_fault_stop_rows(sl.h, rows);
  }
  return SHO_OK;
}

int sho_fault_hold(sho_server* s, int id, int hold) {
  if (!s) return SHO_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->systems.find(id);
    if (it == s->systems.end()) return SHO_ERR_STATE;
    it->second.held = hold != 0;
  }
  s->cv_work.notify_all();
  return SHO_OK;
}

int sho_server_get_stats(sho_server* s, sho_server_stats* out) {
  if (!s || !out) return SHO_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->p50_ms = percentile(s->lat_ms, 0.50);
  out->p99_ms = percentile(s->lat_ms, 0.99);
  double sum = 0.0, mx = 0.0;
  for (double v : s->lat_ms) {
    sum += v;
    mx = std::max(mx, v);
  }
  out->mean_ms = s->lat_ms.empty() ? 0.0 : sum / (double)s->lat_ms.size();
  out->max_ms = mx;
  out->busy_seconds = s->t_first >= 0.0 ? std::max(0.0, s->t_last - s->t_first) : 0.0;
  out->algorithmic_bytes = s->bytes_done;
  out->gbs = out->busy_seconds > 0.0 ? s->bytes_done / out->busy_seconds / 1e9 : 0.0;
  out->resident_bytes = s->resident;
  out->workspace_bytes = s->workspaces();
  out->peak_bytes = s->peak;
  out->max_inflight = s->max_inflight;
  return SHO_OK;
}

int sho_server_reset_stats(sho_server* s) {
  if (!s) return SHO_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->submitted = s->completed = s->failed = 0;
  s->lat_ms.clear();
  s->t_first = -1.0;
  s->t_last = 0.0;
  s->bytes_done = 0.0;
  s->max_inflight = s->inflight;
  s->peak = s->resident + s->workspaces();
  return SHO_OK;
}

}  // extern "C"
