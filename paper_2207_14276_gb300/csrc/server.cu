// Continuous-batching request server over the batched evaluation.
//
// Requests (gas-phase molecules, or new solute coordinates for a registered
// resident solvated box, as lambda windows and replicas issue them) arrive on
// any host thread and join one FIFO queue.  Each of n_lanes lanes owns a
// handle clone (its own work arena, reserved up front), a CUDA stream, device
// and pinned host staging buffers, and a worker thread.  A free lane takes
// every queued request that fits its reserved capacity (atoms and systems:
// the admission by device-memory footprint), stages the inputs with one
// host-to-device copy, runs one batched evaluation, copies energies and forces
// back and completes the requests.  Requests that arrive while lanes are busy
// wait only until a lane frees; lanes run concurrently on separate streams, so
// batches overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/nnp.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxResidents = 256;

struct Resident {
  int64_t n = 0;
  float* coords = nullptr;     // device [n,3]
  uint8_t* species = nullptr;  // device [n]
  uint8_t* mask = nullptr;     // device [n] or null
  double box[3] = {0, 0, 0};
  int periodic = 0;
};

struct Req {
  uint64_t ticket = 0;
  nnp_request_t r{};
  int64_t n_in = 0;            // atoms the evaluation processes
  Clock::time_point t_submit;
  Clock::time_point t_done;
  int status = NNP_PENDING;
  bool done = false;
};

struct Lane {
  nnp_handle* h = nullptr;
  cudaStream_t st = nullptr;
  std::thread th;
  // device buffers
  float* d_xyz = nullptr;
  uint8_t* d_sp = nullptr;
  uint8_t* d_mask = nullptr;
  float* d_f = nullptr;
  double* d_e = nullptr;
  // pinned host staging
  float* h_xyz = nullptr;
  uint8_t* h_sp = nullptr;
  uint8_t* h_mask = nullptr;
  float* h_f = nullptr;
  double* h_e = nullptr;
  std::atomic<long long> batches{0}, requests{0};
};

}  // namespace

struct nnp_server {
  const nnp_handle* model = nullptr;
  int device = 0;
  int max_atoms = 0, max_systems = 0;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::vector<Resident> residents;   // reserved up front: never reallocated
  std::atomic<int> n_residents{0};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::string error;
};

namespace {

int set_err(nnp_server* s, int code, const std::string& m) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->error = m;
  return code;
}

// take every queued request that fits the lane (FIFO, stop at the first misfit)
std::vector<Req*> take_batch(nnp_server* s, std::unique_lock<std::mutex>& lk) {
  s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
  std::vector<Req*> b;
  int64_t atoms = 0;
  while (!s->queue.empty() && (int)b.size() < s->max_systems) {
    Req* q = s->queue.front();
    if (atoms + q->n_in > s->max_atoms && !b.empty()) break;
    atoms += q->n_in;
    b.push_back(q);
    s->queue.pop_front();
  }
  return b;
}

void complete(nnp_server* s, const std::vector<Req*>& b, int status) {
  const auto now = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Req* q : b) {
      q->status = status;
      q->t_done = now;
      q->done = true;
    }
  }
  s->cv_done.notify_all();
}

void lane_loop(nnp_server* s, Lane* L) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Req*> b;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      b = take_batch(s, lk);
      if (b.empty() && s->stop) return;
    }
    if (b.empty()) continue;
    // stage inputs: standalone systems go through the pinned buffer; resident
    // systems are copied device-to-device and their updated atoms overwritten
    std::vector<nnp_system_t> sys(b.size());
    int64_t off = 0;
    int rc = NNP_OK;
    for (size_t k = 0; k < b.size() && rc == NNP_OK; ++k) {
      const nnp_request_t& r = b[k]->r;
      nnp_system_t& d = sys[k];
      std::memset(&d, 0, sizeof(d));
      d.n_atoms = b[k]->n_in;
      d.coords = L->d_xyz + 3 * off;
      d.forces = L->d_f + 3 * off;
      d.energy = L->d_e + k;
      if (r.resident_id >= 0) {
        const Resident& R = s->residents[r.resident_id];
        if (cudaMemcpyAsync(L->d_xyz + 3 * off, R.coords, (size_t)R.n * 12, cudaMemcpyDeviceToDevice, L->st))
          rc = NNP_ERR_CUDA;
        std::memcpy(L->h_xyz + 3 * off, r.coords, (size_t)r.n_atoms * 12);
        d.species = R.species;
        d.mask = R.mask;
        d.periodic = R.periodic;
        for (int c = 0; c < 3; ++c) d.box[c] = R.box[c];
      } else {
        std::memcpy(L->h_xyz + 3 * off, r.coords, (size_t)r.n_atoms * 12);
        std::memcpy(L->h_sp + off, r.species, (size_t)r.n_atoms);
        if (r.mask) std::memcpy(L->h_mask + off, r.mask, (size_t)r.n_atoms);
        d.species = L->d_sp + off;
        d.mask = r.mask ? L->d_mask + off : nullptr;
        d.periodic = r.periodic;
        for (int c = 0; c < 3; ++c) d.box[c] = r.box[c];
      }
      off += b[k]->n_in;
    }
    // one host-to-device copy per staged array (resident updates are short
    // copies on top of the device-to-device copy of their box)
    off = 0;
    int64_t run_beg = 0;
    for (size_t k = 0; k < b.size() && rc == NNP_OK; ++k) {
      const nnp_request_t& r = b[k]->r;
      if (r.resident_id >= 0) {
        if (off > run_beg) {
          if (cudaMemcpyAsync(L->d_xyz + 3 * run_beg, L->h_xyz + 3 * run_beg, (size_t)(off - run_beg) * 12,
                              cudaMemcpyHostToDevice, L->st) ||
              cudaMemcpyAsync(L->d_sp + run_beg, L->h_sp + run_beg, (size_t)(off - run_beg),
                              cudaMemcpyHostToDevice, L->st) ||
              cudaMemcpyAsync(L->d_mask + run_beg, L->h_mask + run_beg, (size_t)(off - run_beg),
                              cudaMemcpyHostToDevice, L->st))
            rc = NNP_ERR_CUDA;
        }
        if (cudaMemcpyAsync(L->d_xyz + 3 * off, L->h_xyz + 3 * off, (size_t)r.n_atoms * 12,
                            cudaMemcpyHostToDevice, L->st))
          rc = NNP_ERR_CUDA;
        off += b[k]->n_in;
        run_beg = off;
      } else {
        off += b[k]->n_in;
      }
    }
    if (rc == NNP_OK && off > run_beg) {
      if (cudaMemcpyAsync(L->d_xyz + 3 * run_beg, L->h_xyz + 3 * run_beg, (size_t)(off - run_beg) * 12,
                          cudaMemcpyHostToDevice, L->st) ||
          cudaMemcpyAsync(L->d_sp + run_beg, L->h_sp + run_beg, (size_t)(off - run_beg), cudaMemcpyHostToDevice,
                          L->st) ||
          cudaMemcpyAsync(L->d_mask + run_beg, L->h_mask + run_beg, (size_t)(off - run_beg),
                          cudaMemcpyHostToDevice, L->st))
        rc = NNP_ERR_CUDA;
    }
    for (int attempt = 0; attempt < 2 && rc == NNP_OK; ++attempt) {
      rc = nnp_energy_forces_batch(L->h, (int)sys.size(), sys.data(), L->st);
      if (rc == NNP_OK) {
        if (cudaMemcpyAsync(L->h_e, L->d_e, sys.size() * sizeof(double), cudaMemcpyDeviceToHost, L->st) ||
            cudaMemcpyAsync(L->h_f, L->d_f, (size_t)off * 12, cudaMemcpyDeviceToHost, L->st))
          rc = NNP_ERR_CUDA;
      }
      if (rc == NNP_OK) rc = nnp_sync_status(L->h, L->st);
      if (rc != NNP_ERR_CAPACITY) break;
      rc = NNP_OK;  // capacity grown by nnp_sync_status: run the batch again
    }
    if (rc == NNP_OK) {
      off = 0;
      for (size_t k = 0; k < b.size(); ++k) {
        const nnp_request_t& r = b[k]->r;
        *r.energy = L->h_e[k];
        if (r.forces) std::memcpy(r.forces, L->h_f + 3 * off, (size_t)r.n_atoms * 12);
        off += b[k]->n_in;
      }
    }
    L->batches += 1;
    L->requests += (long long)b.size();
    complete(s, b, rc);
  }
}

}  // namespace

extern "C" {

int nnp_server_create(const nnp_handle* model, int n_lanes, int64_t max_batch_atoms, int max_batch_systems,
                      nnp_server** out) {
  if (!model || !out || n_lanes < 1 || n_lanes > 16 || max_batch_atoms < 1 || max_batch_systems < 1)
    return NNP_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<nnp_server> s(new nnp_server);
  s->model = model;
  if (cudaGetDevice(&s->device) != cudaSuccess) return NNP_ERR_CUDA;
  s->max_atoms = (int)std::min<int64_t>(max_batch_atoms, 1 << 28);
  s->max_systems = max_batch_systems;
  s->residents.resize(kMaxResidents);
  const size_t A = (size_t)s->max_atoms;
  for (int l = 0; l < n_lanes; ++l) {
    std::unique_ptr<Lane> L(new Lane);
    int rc = nnp_clone(model, &L->h);
    if (rc) return rc;
    rc = nnp_reserve(L->h, s->max_atoms, max_batch_systems, 0, 0);
    if (rc) { nnp_destroy(L->h); return rc; }
    if (cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking) ||
        cudaMalloc(&L->d_xyz, A * 12) || cudaMalloc(&L->d_sp, A) || cudaMalloc(&L->d_mask, A) ||
        cudaMalloc(&L->d_f, A * 12) || cudaMalloc(&L->d_e, (size_t)max_batch_systems * 8) ||
        cudaMallocHost(&L->h_xyz, A * 12) || cudaMallocHost(&L->h_sp, A) ||
        cudaMallocHost(&L->h_mask, A) || cudaMallocHost(&L->h_f, A * 12) ||
        cudaMallocHost(&L->h_e, (size_t)max_batch_systems * 8)) {
      cudaGetLastError();
      nnp_destroy(L->h);
      return NNP_ERR_OOM;
    }
    s->lanes.push_back(std::move(L));
  }
  nnp_server* raw = s.release();
  for (auto& L : raw->lanes) {
    Lane* lp = L.get();
    L->th = std::thread([raw, lp] { lane_loop(raw, lp); });
  }
  *out = raw;
  return NNP_OK;
}

void nnp_server_destroy(nnp_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& L : s->lanes)
    if (L->th.joinable()) L->th.join();
  for (auto& L : s->lanes) {
    cudaStreamSynchronize(L->st);
    cudaFree(L->d_xyz); cudaFree(L->d_sp); cudaFree(L->d_mask); cudaFree(L->d_f); cudaFree(L->d_e);
    cudaFreeHost(L->h_xyz); cudaFreeHost(L->h_sp); cudaFreeHost(L->h_mask); cudaFreeHost(L->h_f);
    cudaFreeHost(L->h_e);
    cudaStreamDestroy(L->st);
    nnp_destroy(L->h);
  }
  for (int i = 0; i < s->n_residents.load(); ++i) {
    Resident& R = s->residents[i];
    cudaFree(R.coords); cudaFree(R.species); cudaFree(R.mask);
  }
  delete s;
}

int nnp_server_register(nnp_server* s, int64_t n_atoms, const float* coords_h, const uint8_t* species_h,
                        const uint8_t* mask_h, const double* box_host, int* resident_id) {
  if (!s || n_atoms < 1 || !coords_h || !species_h || !resident_id) return NNP_ERR_ARG;
  if (n_atoms > s->max_atoms) return set_err(s, NNP_ERR_OOM, "resident system larger than a lane's batch");
  Resident R;
  R.n = n_atoms;
  if (cudaMalloc(&R.coords, (size_t)n_atoms * 12) || cudaMalloc(&R.species, (size_t)n_atoms) ||
      (mask_h && cudaMalloc(&R.mask, (size_t)n_atoms))) {
    cudaGetLastError();
    cudaFree(R.coords); cudaFree(R.species);
    return NNP_ERR_OOM;
  }
  if (cudaMemcpy(R.coords, coords_h, (size_t)n_atoms * 12, cudaMemcpyHostToDevice) ||
      cudaMemcpy(R.species, species_h, (size_t)n_atoms, cudaMemcpyHostToDevice) ||
      (mask_h && cudaMemcpy(R.mask, mask_h, (size_t)n_atoms, cudaMemcpyHostToDevice)))
    return NNP_ERR_CUDA;
  R.periodic = box_host != nullptr;
  for (int c = 0; c < 3; ++c) R.box[c] = box_host ? box_host[c] : 0.0;
  std::lock_guard<std::mutex> lk(s->mu);
  const int id = s->n_residents.load();
  if (id >= kMaxResidents) {
    cudaFree(R.coords); cudaFree(R.species); cudaFree(R.mask);
    s->error = "too many resident systems";
    return NNP_ERR_ARG;
  }
  s->residents[id] = R;
  s->n_residents.store(id + 1);
  *resident_id = id;
  return NNP_OK;
}

int nnp_server_submit(nnp_server* s, const nnp_request_t* r, uint64_t* ticket) {
  if (!s || !r || !ticket || !r->energy || r->n_atoms < 0 || (r->n_atoms > 0 && !r->coords))
    return NNP_ERR_ARG;
  std::unique_ptr<Req> q(new Req);
  q->r = *r;
  if (r->resident_id >= 0) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->resident_id >= s->n_residents.load()) return NNP_ERR_ARG;
    if (r->n_atoms > s->residents[r->resident_id].n) return NNP_ERR_ARG;
    q->n_in = s->residents[r->resident_id].n;
  } else {
    if (r->n_atoms > 0 && !r->species) return NNP_ERR_ARG;
    q->n_in = r->n_atoms;
  }
  if (q->n_in > s->max_atoms) return set_err(s, NNP_ERR_OOM, "request larger than a lane's batch capacity");
  q->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    *ticket = q->ticket;
    s->queue.push_back(q.get());
    s->reqs[q->ticket] = std::move(q);
  }
  s->cv_work.notify_one();
  return NNP_OK;
}

int nnp_server_poll(nnp_server* s, uint64_t ticket, int wait, double* latency_s) {
  if (!s) return NNP_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return NNP_ERR_ARG;
  Req* q = it->second.get();
  if (!q->done) {
    if (!wait) return NNP_PENDING;
    s->cv_done.wait(lk, [&] { return q->done; });
  }
  const int st = q->status;
  if (latency_s) *latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
  s->reqs.erase(it);
  return st;
}

int nnp_server_stats(nnp_server* s, long long* batches, long long* requests) {
  if (!s) return NNP_ERR_ARG;
  long long b = 0, r = 0;
  for (auto& L : s->lanes) { b += L->batches; r += L->requests; }
  if (batches) *batches = b;
  if (requests) *requests = r;
  return NNP_OK;
}

}  // extern "C"
