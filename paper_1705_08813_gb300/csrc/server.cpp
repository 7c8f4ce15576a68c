// Request loop for operator-apply and pressure-solve jobs of different meshes and degrees.
//
// Jobs are admitted as worker slots and device memory free up: a job needs a resident mesh with
// the job's parameters (meshes and their solver state stay on the device between jobs and are
// reused; at most one worker uses a mesh instance at a time, further instances are created while
// the HBM budget allows, idle meshes are evicted least-recently-used when it does not). Each
// worker thread owns a CUDA stream, so the work of concurrent jobs overlaps on the device.
//
// Continuous batching of solves: a worker that takes a mixed-precision solve on a channel mesh
// drives a block solve on that mesh (batch.cu). Between refinement rounds it admits queued solves
// with the same mesh parameters and multigrid settings into free columns (up to 8), and every
// column that converges is reported and frees its column for the next request, so requests that
// arrive while others are on the GPU join the running block. Results do not depend on what else is
// running: a column's arithmetic is the same alone and in any block (per-column reductions, no
// shared scratch between jobs, deterministic kernels).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dgw_internal.h"
#include "solver.h"

namespace {

using clock_type = std::chrono::steady_clock;

struct MeshSlot {
  dgw_mesh_params params;
  dgw_mesh_t mesh = nullptr;
  size_t bytes = 0;
  bool busy = false;
  clock_type::time_point last_used;
  int batch_room = 0;   // free columns of the block solve running on this mesh (0: none running)
  int batch_cheb = 0;
};

struct JobRec {
  long ticket;
  dgw_job job;
  dgw_status status = DGW_EBUSY;   // DGW_EBUSY while queued or running
  dgw_solve_info info{};
  clock_type::time_point t_submit, t_start, t_done;
  bool started = false, done = false;
  const dgw_mesh *in_batch = nullptr;   // the mesh whose block solve runs this job
};

bool same_params(const dgw_mesh_params &a, const dgw_mesh_params &b) {
  return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.degree == b.degree && a.enrich_l == b.enrich_l &&
         a.q_wall == b.q_wall && a.geometry == b.geometry && a.wall_law == b.wall_law && a.n_layers == b.n_layers &&
         a.lx == b.lx && a.ly == b.ly && a.lz == b.lz && a.stretch_gamma == b.stretch_gamma && a.nu == b.nu &&
         a.tau_w == b.tau_w && a.precision_mask == b.precision_mask && a.full_quadrature == b.full_quadrature;
}

// Device bytes a job needs beyond its caller-owned vectors: the mesh and, for solves, the CG
// workspace and an upper bound of the multigrid hierarchy (levels shrink by 8).
size_t footprint_estimate(const dgw_mesh_params &p, int kind) {
  const size_t n1 = (size_t)p.degree + 1, nc = (size_t)p.nx * p.ny * p.nz;
  const size_t np = nc * n1 * n1 * n1;
  const size_t ne = (size_t)2 * p.n_layers * p.nx * p.nz;
  const size_t qi = (3 * (size_t)p.degree) / 2 + 1, qw = p.q_wall > 0 ? (size_t)p.q_wall : 8;
  size_t mesh = np * 8 * 2 + nc * 16 + ne * (qi * qi * qw + 6 * qw * qi) * 8 * 12 + (1 << 20);
  if (kind == DGW_JOB_SOLVE) {
    mesh += np * 8 * 6 + np * 8 * 8 * 8 / 7;   // CG vectors + MG levels (FP64 bound)
    mesh += (size_t)dgw::kBatchMax * np * 96;  // block solve: 4 FP64 + 4 FP32 columns, FP32 levels
  }
  return mesh;
}

}  // namespace

struct dgw_server {
  size_t budget;
  int workers_n;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<long> queue;                      // tickets waiting for a slot
  std::map<long, std::unique_ptr<JobRec>> jobs;
  std::list<MeshSlot> meshes;
  size_t used = 0;
  long next_ticket = 1;
  bool stopping = false;
  int running = 0;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;

  // Try to reserve a resident mesh for the job (caller holds mu). Returns nullptr if none can be
  // had now; sets *fatal when the job can never fit the budget.
  MeshSlot *reserve(const dgw_job &j, bool *fatal) {
    *fatal = false;
    for (auto &m : meshes)
      if (!m.busy && same_params(m.params, j.mesh)) {
        m.busy = true;
        return &m;
      }
    const size_t need = footprint_estimate(j.mesh, j.kind);
    if (need > budget) { *fatal = true; return nullptr; }
    // evict idle meshes, least recently used first, until the new one fits
    while (used + need > budget) {
      auto victim = meshes.end();
      for (auto it = meshes.begin(); it != meshes.end(); ++it)
        if (!it->busy && (victim == meshes.end() || it->last_used < victim->last_used)) victim = it;
      if (victim == meshes.end()) return nullptr;   // wait for running jobs to release memory
      dgw_mesh_destroy(victim->mesh);
      used -= victim->bytes;
      meshes.erase(victim);
    }
    MeshSlot s;
    s.params = j.mesh;
    s.busy = true;
    s.bytes = need;
    s.mesh = nullptr;   // created by the worker outside the lock
    used += need;
    meshes.push_back(s);
    return &meshes.back();
  }

  static bool batchable(const dgw_job &j) {
    return j.kind == DGW_JOB_SOLVE && j.opts.mode == 1 && j.mesh.geometry == 0 && (j.mesh.precision_mask & 2);
  }
  static bool same_batch(const dgw_job &a, const dgw_job &b) {
    return same_params(a.mesh, b.mesh) && a.opts.cheb_degree == b.opts.cheb_degree;
  }

  // Block solve on the mesh of r's job: admits r, then, between refinement rounds, every queued
  // solve that fits the block, until no column is left. Returns false (nothing done) when the mesh
  // cannot host a block (its multigrid needs the iterative coarse solve).
  bool run_batch(JobRec *r, MeshSlot *slot, cudaStream_t s) {
    dgw_mesh *M = slot->mesh;
    // r is finished after its first rounds and its record freed once the client polls it: keep
    // what later admissions compare against
    const dgw_job key = r->job;
    const int cheb = key.opts.cheb_degree > 0 ? key.opts.cheb_degree : 5;
    if (M->batch && M->batch_cheb != cheb) { dgw::batch_destroy(M->batch); M->batch = nullptr; }
    if (!M->batch) {
      dgw::Batch *B = nullptr;
      if (dgw::batch_create(M, dgw::kBatchMax, cheb, &B) != cudaSuccess) return false;
      M->batch = B;
      M->batch_cheb = cheb;
    }
    dgw::Batch *B = M->batch;
    std::vector<JobRec *> incoming{r};
    std::vector<dgw::BatchColumn> done;
    for (;;) {
      for (JobRec *q : incoming) {
        dgw::BatchColumn c;
        c.b_in = (const double *)q->job.in;
        c.p_out = (double *)q->job.out;
        c.tag = q->ticket;
        c.rtol = q->job.opts.rtol;
        c.max_iter = q->job.opts.max_iter;
        if (dgw::batch_admit(B, c, s) != cudaSuccess) {
          (void)cudaGetLastError();   // handled here: must not surface in a later call of this thread
          finish(q, DGW_ECUDA, dgw_solve_info{});
        }
      }
      incoming.clear();
      if (dgw::batch_active(B) == 0) break;
      done.clear();
      const cudaError_t e = dgw::batch_round(B, done);
      if (e != cudaSuccess) {
        // a failed round: every column of the block fails, and the block is rebuilt on next use
        (void)cudaGetLastError();
        dgw::batch_destroy(M->batch);
        M->batch = nullptr;
        std::lock_guard<std::mutex> lock(mu);
        for (auto &kv : jobs)
          if (kv.second->started && !kv.second->done && kv.second->in_batch == M) fail_locked(kv.second.get(), DGW_ECUDA);
        slot->batch_room = 0;
        return true;
      }
      std::lock_guard<std::mutex> lock(mu);
      for (const dgw::BatchColumn &c : done) {
        auto it = jobs.find(c.tag);
        if (it == jobs.end()) continue;
        dgw_solve_info inf{};
        inf.iterations = c.iterations;
        inf.rel_residual = c.rel_residual;
        inf.ms = (float)std::chrono::duration<double, std::milli>(clock_type::now() - c.t_admit).count();
        finish_locked(it->second.get(), c.status, inf);
      }
      // continuous batching: queued solves on this mesh join the block in its free columns
      int room = dgw::kBatchMax - dgw::batch_active(B);
      slot->batch_cheb = cheb;
      for (auto qi = queue.begin(); qi != queue.end() && room > 0;) {
        JobRec *q = jobs[*qi].get();
        if (batchable(q->job) && same_batch(q->job, key)) {
          q->started = true;
          q->t_start = clock_type::now();
          q->in_batch = M;
          ++running;
          incoming.push_back(q);
          qi = queue.erase(qi);
          --room;
        } else {
          ++qi;
        }
      }
      // other workers leave matching solves to this block while it has room
      slot->batch_room = (dgw::batch_active(B) + (int)incoming.size() > 0) ? std::max(room, 0) : 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    slot->batch_room = 0;
    return true;
  }

  // a running block solve with free columns will take this job at its next round
  bool block_will_take(const dgw_job &j) const {
    if (!batchable(j)) return false;
    const int cheb = j.opts.cheb_degree > 0 ? j.opts.cheb_degree : 5;
    for (const auto &m : meshes)
      if (m.busy && m.batch_room > 0 && m.batch_cheb == cheb && same_params(m.params, j.mesh)) return true;
    return false;
  }

  void finish_locked(JobRec *r, dgw_status st, const dgw_solve_info &inf) {
    r->status = st;
    r->info = inf;
    r->t_done = clock_type::now();
    r->done = true;
    --running;
    cv_done.notify_all();
    cv_work.notify_all();
  }
  void fail_locked(JobRec *r, dgw_status st) { finish_locked(r, st, dgw_solve_info{}); }
  void finish(JobRec *r, dgw_status st, const dgw_solve_info &inf) {
    std::lock_guard<std::mutex> lock(mu);
    finish_locked(r, st, inf);
  }

  void run_job(JobRec *r, MeshSlot *slot, cudaStream_t s) {
    (void)cudaGetLastError();   // an error an earlier job of this thread handled is not this job's
    dgw_status st = DGW_OK;
    if (!slot->mesh) {
      st = dgw_mesh_create(&slot->params, s, &slot->mesh);
      if (st == DGW_OK) {
        size_t b = 0;
        dgw_mesh_info(slot->mesh, nullptr, nullptr, nullptr, &b);
        (void)b;
      }
    }
    const dgw_job &j = r->job;
    if (st == DGW_OK && batchable(j)) {
      {
        std::lock_guard<std::mutex> lock(mu);
        r->in_batch = slot->mesh;
      }
      if (run_batch(r, slot, s)) {   // r and every job that joined the block are reported
        std::lock_guard<std::mutex> lock(mu);
        slot->busy = false;
        slot->last_used = clock_type::now();
        cv_work.notify_all();
        return;
      }
    }
    if (st == DGW_OK) {
      switch (j.kind) {
        case DGW_JOB_SOLVE:
          st = dgw_pressure_solve(slot->mesh, (const double *)j.in, (double *)j.out, &j.opts, &r->info, s);
          break;
        case DGW_JOB_LAPLACE: st = dgw_apply_laplace(slot->mesh, j.prec, j.in, j.out, s); break;
        case DGW_JOB_DIVERGENCE: st = dgw_apply_divergence(slot->mesh, (const double *)j.in, (double *)j.out, s); break;
        case DGW_JOB_CONVECTIVE: st = dgw_apply_convective(slot->mesh, j.prec, j.in, j.out, s); break;
        case DGW_JOB_VISCOUS:
          if (j.aux) st = dgw_update_eddy_viscosity(slot->mesh, j.aux, s);
          if (st == DGW_OK) st = dgw_apply_viscous(slot->mesh, j.prec, j.in, j.out, s);
          break;
        default: st = DGW_EINVAL;
      }
      if (st == DGW_OK && j.kind != DGW_JOB_SOLVE) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = DGW_ECUDA;
      }
    }
    std::lock_guard<std::mutex> lock(mu);
    if (st != DGW_OK && !slot->mesh) {
      // creation failed: drop the slot and its reservation
      for (auto it = meshes.begin(); it != meshes.end(); ++it)
        if (&*it == slot) { used -= it->bytes; meshes.erase(it); break; }
    } else {
      slot->busy = false;
      slot->last_used = clock_type::now();
    }
    r->status = st;
    r->t_done = clock_type::now();
    r->done = true;
    --running;
    cv_done.notify_all();
    cv_work.notify_all();
  }

  void worker_main(int w) {
    cudaStream_t s = streams[w];
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
      JobRec *pick = nullptr;
      MeshSlot *slot = nullptr;
      bool rescan = false;
      for (auto it = queue.begin(); it != queue.end(); ++it) {
        JobRec *r = jobs[*it].get();
        if (block_will_take(r->job)) continue;
        bool fatal = false;
        slot = reserve(r->job, &fatal);
        if (fatal) {   // can never fit the budget: fail it and look again
          r->status = DGW_ENOMEM;
          r->done = true;
          r->t_done = clock_type::now();
          queue.erase(it);
          cv_done.notify_all();
          rescan = true;
          break;
        }
        if (slot) {
          pick = r;
          queue.erase(it);
          break;
        }
      }
      if (rescan) continue;
      if (pick) {
        pick->started = true;
        pick->t_start = clock_type::now();
        ++running;
        lock.unlock();
        run_job(pick, slot, s);
        lock.lock();
        continue;
      }
      if (stopping) return;
      cv_work.wait_for(lock, std::chrono::milliseconds(50));
    }
  }
};

extern "C" {

dgw_status dgw_server_create(size_t hbm_budget, int max_inflight, dgw_server_t *out) {
  if (!out || max_inflight < 1 || max_inflight > 64 || hbm_budget == 0)
    return dgw::set_error(DGW_EINVAL, "dgw_server_create: need out, 1 <= max_inflight <= 64, hbm_budget > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return dgw::set_error(DGW_ECUDA, "dgw_server_create: no CUDA device");
  int dev = 0;
  cudaGetDevice(&dev);
  auto *S = new dgw_server();
  S->budget = hbm_budget;
  S->workers_n = max_inflight;
  for (int w = 0; w < max_inflight; ++w) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : S->streams) cudaStreamDestroy(x);
      delete S;
      return dgw::set_error(DGW_ECUDA, "dgw_server_create: stream creation failed");
    }
    S->streams.push_back(st);
  }
  for (int w = 0; w < max_inflight; ++w)
    S->workers.emplace_back([S, w, dev]() {
      cudaSetDevice(dev);
      S->worker_main(w);
    });
  *out = S;
  return DGW_OK;
}

dgw_status dgw_submit(dgw_server_t S, const dgw_job *job, long *ticket) {
  if (!S || !job || !ticket) return dgw::set_error(DGW_EINVAL, "dgw_submit: null argument");
  if (job->kind < DGW_JOB_SOLVE || job->kind > DGW_JOB_VISCOUS || !job->in || !job->out)
    return dgw::set_error(DGW_EINVAL, "dgw_submit: bad job kind or null buffers");
  if (job->mesh.degree < 1 || job->mesh.degree > 5 || job->mesh.nx < 1 || job->mesh.ny < 1 || job->mesh.nz < 1)
    return dgw::set_error(DGW_EINVAL, "dgw_submit: bad mesh parameters");
  auto r = std::make_unique<JobRec>();
  r->job = *job;
  r->t_submit = clock_type::now();
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->stopping) return dgw::set_error(DGW_EINVAL, "dgw_submit: server is shutting down");
  r->ticket = S->next_ticket++;
  *ticket = r->ticket;
  S->queue.push_back(r->ticket);
  S->jobs[r->ticket] = std::move(r);
  S->cv_work.notify_one();
  return DGW_OK;
}

dgw_status dgw_poll(dgw_server_t S, long ticket, dgw_status *job_status, dgw_solve_info *info, double *latency_ms) {
  if (!S || !job_status) return dgw::set_error(DGW_EINVAL, "dgw_poll: null argument");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return dgw::set_error(DGW_EINVAL, "dgw_poll: unknown ticket");
  JobRec *r = it->second.get();
  if (!r->done) {
    *job_status = DGW_EBUSY;
    return DGW_EBUSY;
  }
  *job_status = r->status;
  if (info) *info = r->info;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  S->jobs.erase(it);   // a completed ticket is reported once
  return DGW_OK;
}

dgw_status dgw_server_destroy(dgw_server_t S, int timeout_ms) {
  if (!S) return dgw::set_error(DGW_EINVAL, "dgw_server_destroy: null server");
  dgw_status result = DGW_OK;
  {
    std::unique_lock<std::mutex> lock(S->mu);
    // cancel what has not started
    for (long t : S->queue) {
      JobRec *r = S->jobs[t].get();
      r->status = DGW_ETIMEOUT;
      r->done = true;
    }
    S->queue.clear();
    S->stopping = true;
    S->cv_work.notify_all();
    const auto deadline = clock_type::now() + std::chrono::milliseconds(timeout_ms > 0 ? timeout_ms : 0);
    while (S->running > 0) {
      if (S->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && S->running > 0) {
        result = DGW_ETIMEOUT;
        break;
      }
    }
  }
  if (result == DGW_ETIMEOUT) {
    // running jobs still own streams and meshes: leave the server alive rather than free under them
    return dgw::set_error(DGW_ETIMEOUT, "dgw_server_destroy: running jobs did not finish in time");
  }
  for (auto &t : S->workers) t.join();
  for (auto &m : S->meshes)
    if (m.mesh) dgw_mesh_destroy(m.mesh);
  for (auto st : S->streams) cudaStreamDestroy(st);
  delete S;
  return DGW_OK;
}

dgw_status dgw_server_stats(dgw_server_t S, int *queued, int *running, int *resident_meshes, size_t *reserved_bytes) {
  if (!S) return dgw::set_error(DGW_EINVAL, "dgw_server_stats: null server");
  std::lock_guard<std::mutex> lock(S->mu);
  if (queued) *queued = (int)S->queue.size();
  if (running) *running = S->running;
  if (resident_meshes) *resident_meshes = (int)S->meshes.size();
  if (reserved_bytes) *reserved_bytes = S->used;
  return DGW_OK;
}

}  // extern "C"
