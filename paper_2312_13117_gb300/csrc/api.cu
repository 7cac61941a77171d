// C ABI of libpmcim and the host-side driver of pmCIMb (Sec. 3.2).
//
// The driver turns a list of disks into a list of nodes (one linear system each),
// runs the node solves in HBM-sized waves, reduces the solves per disk, gates
// disks by the indicator, runs Beyn's extraction on candidates, splits saturated
// disks into four children (pmCIMa's quadrisection geometry, Sec. 3.1) and
// verifies the surviving values. All arithmetic of the method runs in the CUDA
// kernels; the host only builds work lists, moves small results and sorts.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pmcim_internal.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CU(expr)                                                                              \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess)                                                                    \
      return fail(_e == cudaErrorMemoryAllocation ? PMCIM_ENOMEM : PMCIM_ECUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(_e), __FILE__, __LINE__);                         \
  } while (0)

#define CHK(expr)               \
  do {                          \
    int _r = (expr);            \
    if (_r != PMCIM_OK) return _r; \
  } while (0)

// Growable device buffer owned by a problem handle.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  // grow to at least `bytes`, keeping the first `keep` bytes
  cudaError_t grow_keep(size_t bytes, size_t keep, cudaStream_t s) {
    if (bytes <= cap) return cudaSuccess;
    size_t nc = std::max(bytes, 2 * cap);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, nc);
    if (e != cudaSuccess) return e;
    if (p && keep) {
      e = cudaMemcpyAsync(q, p, keep, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { cudaFree(q); return e; }
    }
    if (p) cudaFree(p);
    p = q;
    cap = nc;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Upper bound on the solution buffer of one wave (node solves kept before reduction).
constexpr size_t kWaveBytes = size_t(4) << 30;
// Upper bound on the per-CTA factorisation workspaces.
constexpr size_t kSlotBytes = size_t(24) << 30;
// Refinement stops when the estimated remaining error of X (max norm) is below
// this fraction of |X|: 1e-11 keeps Beyn's eigenvalues within about 1e-14 of
// the FP64 ones on the delay workload (simulated FP32 LU + FP64 refinement).
constexpr double kIrTol = 1e-11;

// Copy results to a caller buffer that may live on the host or the device.
int copy_out(void* dst, const void* src, size_t bytes) {
  if (!bytes) return PMCIM_OK;
  CU(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
  return PMCIM_OK;
}

// ---- launch accounting ----------------------------------------------------
struct Prof {
  std::mutex mu;
  bool on = false;
  int64_t launches[PMCIM_K_COUNT] = {};
  double ms[PMCIM_K_COUNT] = {};
  double phase[8] = {};
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t cur_begin[PMCIM_K_COUNT] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
Prof& prof() {
  static Prof* p = new Prof();
  return *p;
}

}  // namespace

bool prof_on();
void prof_add_phases(const unsigned long long* c, int slots);

void prof_begin(int kind, cudaStream_t s) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.launches[kind] += 1;
  if (!P.on) return;
  cudaEvent_t e = P.get();
  cudaEventRecord(e, s);
  P.cur_begin[kind] = e;
}

void prof_end(int kind, cudaStream_t s) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  if (!P.on || !P.cur_begin[kind]) return;
  cudaEvent_t e = P.get();
  cudaEventRecord(e, s);
  P.pending.push_back({kind, P.cur_begin[kind], e});
  P.cur_begin[kind] = nullptr;
}

bool prof_on() {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  return P.on;
}

void prof_add_phases(const unsigned long long* c, int slots) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  for (int b = 0; b < slots; ++b)
    for (int q = 0; q < 8; ++q) P.phase[q] += (double)c[(size_t)b * 8 + q];
}

void prof_flush() {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  for (auto& q : P.pending) {
    float t = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&t, q.a, q.b) == cudaSuccess)
      P.ms[q.kind] += t;
    P.pool.push_back(q.a);
    P.pool.push_back(q.b);
  }
  P.pending.clear();
}

struct pmcim_problem_s {
  int n = 0, K = 0;
  ProblemDesc desc{};
  double2* dA = nullptr;
  int device = 0;
  // workspaces, reused across calls
  DevBuf work, piv, X, node_info, regions, node_region, V;
  DevBuf C0, C1, pf_half, pf_abs, ind, pf_norm, pf_scale, cand;
  DevBuf bslot, bregion, bwork, bsigma, bp, blam, bvecs, bkept, bstatus;
  DevBuf vlam, vsig, vacc, vwork, vvec, vpiv;
  DevBuf gsrc, gdst, gperm, phase;
};

namespace {

struct HostRegion {
  double cre, cim, r;
  int N;
  int depth;
  int root;  // index of the caller's disk this one descends from
};

int check_options(const pmcim_options* opt) {
  if (!opt) return fail(PMCIM_EINVAL, "options pointer is NULL");
  if (!(opt->tol_ind >= 0.0) || !(opt->tol_svd >= 0.0) || !(opt->tol_verify >= 0.0))
    return fail(PMCIM_EINVAL, "tolerances must be non-negative");
  if (opt->precision != PMCIM_PREC_FP64 && opt->precision != PMCIM_PREC_FP32_IR)
    return fail(PMCIM_EINVAL, "unknown precision %d", opt->precision);
  if (opt->max_split_depth < 0 || opt->max_split_depth > 30) return fail(PMCIM_EINVAL, "max_split_depth out of range");
  if (opt->precision == PMCIM_PREC_FP32_IR && (opt->max_ir_sweeps < 1 || opt->max_ir_sweeps > 10))
    return fail(PMCIM_EINVAL, "max_ir_sweeps must be 1..10");
  return PMCIM_OK;
}

int check_regions(int R, const pmcim_region* reg, int l, int n) {
  if (R < 0) return fail(PMCIM_EINVAL, "negative region count");
  if (R > 0 && !reg) return fail(PMCIM_EINVAL, "regions pointer is NULL");
  if (l < 1 || l > PMCIM_MAX_L) return fail(PMCIM_EINVAL, "l = %d outside 1..%d", l, PMCIM_MAX_L);
  (void)n;
  for (int g = 0; g < R; ++g) {
    if (reg[g].N < 2 || reg[g].N > 4096 || (reg[g].N & 1))
      return fail(PMCIM_EINVAL, "region %d: N = %d must be even, 2..4096", g, reg[g].N);
    if (!(reg[g].r > 0.0) || !std::isfinite(reg[g].r) || !std::isfinite(reg[g].c_re) || !std::isfinite(reg[g].c_im))
      return fail(PMCIM_EINVAL, "region %d: bad centre or radius", g);
  }
  return PMCIM_OK;
}

cudaStream_t stream_of(const pmcim_options* opt) { return reinterpret_cast<cudaStream_t>(opt->cuda_stream); }

// Copy the probe block to the device once per call.
int upload_V(pmcim_problem p, int l, const double* V, cudaStream_t s) {
  if (!V) return fail(PMCIM_EINVAL, "V is NULL");
  const size_t bytes = (size_t)p->n * l * sizeof(double2);
  CU(p->V.ensure(bytes));
  CU(cudaMemcpyAsync(p->V.p, V, bytes, cudaMemcpyDefault, s));
  return PMCIM_OK;
}

// Moments of every disk in `regs` into p->C0/C1/pf_half/pf_abs (region-major),
// and per-disk singular-node flags into `singular` (host).
int run_moments(pmcim_problem p, const pmcim_options* opt, const std::vector<HostRegion>& regs, int l,
                std::vector<int>* singular, int64_t* solves, int* fallbacks = nullptr,
                int64_t* sweeps = nullptr) {
  cudaStream_t s = stream_of(opt);
  const int n = p->n;
  const int R = (int)regs.size();
  const size_t nl = (size_t)n * l;
  CU(p->C0.ensure(std::max<size_t>(1, R) * nl * sizeof(double2)));
  CU(p->C1.ensure(std::max<size_t>(1, R) * nl * sizeof(double2)));
  CU(p->pf_half.ensure(std::max<size_t>(1, R) * n * sizeof(double2)));
  CU(p->pf_abs.ensure(std::max<size_t>(1, R) * n * sizeof(double)));
  if (singular) singular->assign(R, 0);
  if (R == 0) return PMCIM_OK;

  const bool mixed = opt->precision == PMCIM_PREC_FP32_IR;
  const size_t slot_bytes = mixed ? mixed_slot_bytes(n, l) : (size_t)n * (n + l) * sizeof(double2);
  size_t total_nodes = 0;
  for (const HostRegion& h : regs) total_nodes += (size_t)h.N;
  const int slots = (int)std::max<size_t>(
      1, std::min<size_t>(std::min<size_t>(factor_slots_fp64(n, l), kSlotBytes / slot_bytes), total_nodes));
  CU(p->work.ensure((size_t)slots * slot_bytes));
  CU(p->piv.ensure((size_t)slots * n * sizeof(int32_t)));

  // waves of whole disks whose solutions fit the wave buffer
  const size_t per_node = nl * sizeof(double2);
  int g0 = 0;
  std::vector<RegionDev> rd;
  std::vector<int32_t> node_region;
  std::vector<int32_t> info;
  while (g0 < R) {
    int g1 = g0;
    size_t nodes = 0;
    while (g1 < R && (g1 == g0 || (nodes + regs[g1].N) * per_node <= kWaveBytes) && g1 - g0 < 65535) {
      nodes += regs[g1].N;
      ++g1;
    }
    rd.resize(g1 - g0);
    node_region.resize(nodes);
    int off = 0;
    for (int g = g0; g < g1; ++g) {
      RegionDev& d = rd[g - g0];
      d.cre = regs[g].cre;
      d.cim = regs[g].cim;
      d.r = regs[g].r;
      d.N = regs[g].N;
      d.node_off = off;
      for (int j = 0; j < regs[g].N; ++j) node_region[off + j] = g - g0;
      off += regs[g].N;
    }
    CU(p->X.ensure(std::max<size_t>(1, nodes) * per_node));
    CU(p->node_info.ensure(nodes * sizeof(int32_t)));
    CU(p->regions.ensure(rd.size() * sizeof(RegionDev)));
    CU(p->node_region.ensure(nodes * sizeof(int32_t)));
    CU(cudaMemcpyAsync(p->regions.p, rd.data(), rd.size() * sizeof(RegionDev), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(p->node_region.p, node_region.data(), nodes * sizeof(int32_t), cudaMemcpyHostToDevice, s));

    if (mixed) {
      MixedArgs ma;
      ma.prob = p->desc;
      ma.A = p->dA;
      ma.V = p->V.as<double2>();
      ma.l = l;
      ma.regions = p->regions.as<RegionDev>();
      ma.node_region = p->node_region.as<int32_t>();
      ma.n_nodes = (int)nodes;
      ma.X = p->X.as<double2>();
      ma.node_info = p->node_info.as<int32_t>();
      ma.work = p->work.as<char>();
      ma.slot_bytes = slot_bytes;
      ma.piv = p->piv.as<int32_t>();
      ma.slots = slots;
      ma.max_sweeps = opt->max_ir_sweeps;
      ma.tol_ir = kIrTol;
      ma.phase = nullptr;
      const bool timed = prof_on();
      if (timed) {
        CU(p->phase.ensure((size_t)slots * 8 * sizeof(unsigned long long)));
        CU(cudaMemsetAsync(p->phase.p, 0, (size_t)slots * 8 * sizeof(unsigned long long), s));
        ma.phase = p->phase.as<unsigned long long>();
      }
      prof_begin(PMCIM_K_FACTOR32, s);
      CU(launch_factor_solve_mixed(ma, s));
      prof_end(PMCIM_K_FACTOR32, s);
      if (timed) {
        std::vector<unsigned long long> c((size_t)slots * 8);
        CU(cudaMemcpyAsync(c.data(), p->phase.p, c.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        prof_add_phases(c.data(), slots);
      }
    } else {
      FactorArgs fa;
      fa.prob = p->desc;
      fa.A = p->dA;
      fa.V = p->V.as<double2>();
      fa.l = l;
      fa.regions = p->regions.as<RegionDev>();
      fa.node_region = p->node_region.as<int32_t>();
      fa.n_nodes = (int)nodes;
      fa.X = p->X.as<double2>();
      fa.node_info = p->node_info.as<int32_t>();
      fa.work = p->work.as<double2>();
      fa.piv = p->piv.as<int32_t>();
      fa.slots = slots;
      prof_begin(PMCIM_K_FACTOR, s);
      CU(launch_factor_solve_fp64(fa, s));
      prof_end(PMCIM_K_FACTOR, s);
    }

    ReduceArgs ra;
    ra.X = p->X.as<double2>();
    ra.n = n;
    ra.l = l;
    ra.regions = p->regions.as<RegionDev>();
    ra.R = g1 - g0;
    ra.C0 = p->C0.as<double2>() + (size_t)g0 * nl;
    ra.C1 = p->C1.as<double2>() + (size_t)g0 * nl;
    ra.pf_half = p->pf_half.as<double2>() + (size_t)g0 * n;
    ra.pf_abs = p->pf_abs.as<double>() + (size_t)g0 * n;
    prof_begin(PMCIM_K_REDUCE, s);
    CU(launch_reduce_moments(ra, s));
    prof_end(PMCIM_K_REDUCE, s);

    if (singular) {
      info.resize(nodes);
      CU(cudaMemcpyAsync(info.data(), p->node_info.p, nodes * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      for (int g = g0; g < g1; ++g) {
        const RegionDev& d = rd[g - g0];
        for (int j = 0; j < d.N; ++j) {
          const int v = info[d.node_off + j];
          if (v & 0x00ffffff) (*singular)[g] |= 1;
          if (sweeps) *sweeps += (v >> 24) & 63;
          if (v & (1 << 30)) {
            (*singular)[g] |= 2;
            if (fallbacks) *fallbacks += 1;
          }
        }
      }
    }
    if (solves) *solves += (int64_t)nodes;
    g0 = g1;
  }
  return PMCIM_OK;
}

// Indicator of every disk whose moments are in p->C0 etc.
int run_indicator(pmcim_problem p, const pmcim_options* opt, int R, int l) {
  cudaStream_t s = stream_of(opt);
  CU(p->ind.ensure(std::max(1, R) * sizeof(double)));
  CU(p->pf_norm.ensure(std::max(1, R) * sizeof(double)));
  CU(p->pf_scale.ensure(std::max(1, R) * sizeof(double)));
  CU(p->cand.ensure(std::max(1, R) * sizeof(uint8_t)));
  IndicatorArgs ia;
  ia.C0 = p->C0.as<double2>();
  ia.pf_half = p->pf_half.as<double2>();
  ia.pf_abs = p->pf_abs.as<double>();
  ia.n = p->n;
  ia.l = l;
  ia.R = R;
  ia.tol_ind = opt->tol_ind;
  ia.ind = p->ind.as<double>();
  ia.pf_norm = p->pf_norm.as<double>();
  ia.pf_scale = p->pf_scale.as<double>();
  ia.candidate = p->cand.as<uint8_t>();
  prof_begin(PMCIM_K_INDICATOR, s);
  CU(launch_indicator(ia, s));
  prof_end(PMCIM_K_INDICATOR, s);
  return PMCIM_OK;
}

struct EigOut {
  std::vector<double2> lam;
  std::vector<int> root;
  int n_vecs = 0;  // vectors gathered into p->gdst so far (same order as lam)
};

// pmCIMb step 2 with splitting of saturated disks. `gate_top` applies the
// indicator gate to the caller's disks too (pmcim_solve); children are always gated.
int run_beyn_levels(pmcim_problem p, const pmcim_options* opt, const std::vector<HostRegion>& top, int l,
                    bool gate_top, bool want_vecs, EigOut* out, std::vector<int>* root_status,
                    std::vector<double>* top_ind, pmcim_stats* st) {
  cudaStream_t s = stream_of(opt);
  const int n = p->n;
  const size_t nl = (size_t)n * l;
  std::vector<HostRegion> level = top;
  root_status->assign(top.size(), 0);
  if (top_ind) top_ind->assign(top.size(), 0.0);
  while (!level.empty()) {
    const int R = (int)level.size();
    std::vector<int> singular;
    int64_t solves = 0;
    int fallbacks = 0;
    int64_t sweeps = 0;
    CHK(run_moments(p, opt, level, l, &singular, &solves, &fallbacks, &sweeps));
    if (st) {
      st->ir_fallbacks += fallbacks;
      st->ir_sweeps += sweeps;
    }
    CHK(run_indicator(p, opt, R, l));
    std::vector<double> ind(R);
    std::vector<uint8_t> cflag(R);
    CU(cudaMemcpyAsync(ind.data(), p->ind.p, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(cflag.data(), p->cand.p, R * sizeof(uint8_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (st) {
      st->solves += solves;
      st->regions += R;
    }
    std::vector<int32_t> slot;
    std::vector<RegionDev> crd;
    for (int g = 0; g < R; ++g) {
      const HostRegion& h = level[g];
      if (singular[g] & 1) {
        (*root_status)[h.root] |= PMCIM_RS_SINGULAR_NODE;
        if (st) st->singular_nodes += 1;
      }
      if (singular[g] & 2) (*root_status)[h.root] |= PMCIM_RS_IR_FALLBACK;
      if (h.depth == 0 && top_ind) (*top_ind)[h.root] = ind[g];
      const bool gated = (h.depth > 0) || gate_top;
      if (cflag[g]) (*root_status)[h.root] |= PMCIM_RS_CANDIDATE;
      if (gated && !cflag[g]) continue;
      if (st) st->candidates += 1;
      slot.push_back(g);
      RegionDev d;
      d.cre = h.cre;
      d.cim = h.cim;
      d.r = h.r;
      d.N = h.N;
      d.node_off = 0;
      crd.push_back(d);
    }
    const int m = (int)slot.size();
    std::vector<HostRegion> next;
    if (m > 0) {
      CU(p->bslot.ensure(m * sizeof(int32_t)));
      CU(p->bregion.ensure(m * sizeof(RegionDev)));
      CU(p->bwork.ensure((size_t)m * (2 * nl + 4 * (size_t)l * l) * sizeof(double2)));
      CU(p->bsigma.ensure((size_t)m * l * sizeof(double)));
      CU(p->bp.ensure(m * sizeof(int32_t)));
      CU(p->blam.ensure((size_t)m * l * sizeof(double2)));
      CU(p->bvecs.ensure((size_t)m * nl * sizeof(double2)));
      CU(p->bkept.ensure((size_t)m * l));
      CU(p->bstatus.ensure(m * sizeof(int32_t)));
      CU(cudaMemcpyAsync(p->bslot.p, slot.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      CU(cudaMemcpyAsync(p->bregion.p, crd.data(), m * sizeof(RegionDev), cudaMemcpyHostToDevice, s));
      BeynArgs ba;
      ba.C0 = p->C0.as<double2>();
      ba.C1 = p->C1.as<double2>();
      ba.slot_of = p->bslot.as<int32_t>();
      ba.regions = p->bregion.as<RegionDev>();
      ba.n = n;
      ba.l = l;
      ba.m = m;
      ba.tol_svd = opt->tol_svd;
      ba.work = p->bwork.as<double2>();
      ba.sigma = p->bsigma.as<double>();
      ba.p = p->bp.as<int32_t>();
      ba.lam = p->blam.as<double2>();
      ba.vecs = p->bvecs.as<double2>();
      ba.kept = p->bkept.as<uint8_t>();
      ba.status = p->bstatus.as<int32_t>();
      prof_begin(PMCIM_K_BEYN, s);
      CU(launch_beyn(ba, s));
      prof_end(PMCIM_K_BEYN, s);
      std::vector<int32_t> pv(m), stv(m);
      std::vector<double2> lam((size_t)m * l);
      std::vector<uint8_t> kept((size_t)m * l);
      CU(cudaMemcpyAsync(pv.data(), p->bp.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CU(cudaMemcpyAsync(stv.data(), p->bstatus.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CU(cudaMemcpyAsync(lam.data(), p->blam.p, (size_t)m * l * sizeof(double2), cudaMemcpyDeviceToHost, s));
      CU(cudaMemcpyAsync(kept.data(), p->bkept.p, (size_t)m * l, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      std::vector<int32_t> gsrc;
      for (int c = 0; c < m; ++c) {
        const HostRegion& h = level[slot[c]];
        int bits = stv[c];
        if ((bits & PMCIM_RS_SATURATED) && h.depth < opt->max_split_depth) {
          (*root_status)[h.root] |= PMCIM_RS_SATURATED | PMCIM_RS_SPLIT;
          if (st) st->splits += 1;
          const double rc = h.r / 2.0, d = rc / std::sqrt(2.0);
          const int sx[4] = {1, -1, 1, -1}, sy[4] = {1, 1, -1, -1};
          for (int q = 0; q < 4; ++q)
            next.push_back(HostRegion{h.cre + sx[q] * d, h.cim + sy[q] * d, rc, h.N, h.depth + 1, h.root});
          continue;
        }
        (*root_status)[h.root] |= bits;
        for (int k = 0; k < pv[c]; ++k) {
          if (!kept[(size_t)c * l + k]) continue;
          out->lam.push_back(lam[(size_t)c * l + k]);
          out->root.push_back(h.root);
          gsrc.push_back(c * l + k);
        }
      }
      if (want_vecs && !gsrc.empty()) {
        const int cnt = (int)gsrc.size();
        {
          const size_t vb = (size_t)n * sizeof(double2);
          CU(p->gdst.grow_keep((size_t)(out->n_vecs + cnt) * vb, (size_t)out->n_vecs * vb, s));
          CU(p->gsrc.ensure(cnt * sizeof(int32_t)));
          CU(cudaMemcpyAsync(p->gsrc.p, gsrc.data(), cnt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
          GatherArgs ga;
          ga.vecs = p->bvecs.as<double2>();
          ga.src = p->gsrc.as<int32_t>();
          ga.dst = p->gdst.as<double2>() + (size_t)out->n_vecs * n;
          ga.n = n;
          ga.l = l;
          ga.count = cnt;
          prof_begin(PMCIM_K_GATHER, s);
          CU(launch_gather_vecs(ga, s));
          prof_end(PMCIM_K_GATHER, s);
          CU(cudaStreamSynchronize(s));
        }
        out->n_vecs += cnt;
      }
    }
    level.swap(next);
  }
  return PMCIM_OK;
}

int run_verify(pmcim_problem p, const pmcim_options* opt, const std::vector<double2>& lam,
               std::vector<double>* sig, std::vector<uint8_t>* acc) {
  cudaStream_t s = stream_of(opt);
  const int m = (int)lam.size();
  sig->assign(m, 0.0);
  acc->assign(m, 0);
  if (m == 0) return PMCIM_OK;
  const int n = p->n;
  const int slots = std::min(verify_slots_fp64(n), m);
  CU(p->vlam.ensure(m * sizeof(double2)));
  CU(p->vsig.ensure(m * sizeof(double)));
  CU(p->vacc.ensure(m));
  CU(p->vwork.ensure((size_t)slots * n * n * sizeof(double2)));
  CU(p->vvec.ensure((size_t)slots * 3 * n * sizeof(double2)));
  CU(p->vpiv.ensure((size_t)slots * n * sizeof(int32_t)));
  CU(cudaMemcpyAsync(p->vlam.p, lam.data(), m * sizeof(double2), cudaMemcpyHostToDevice, s));
  VerifyArgs va;
  va.prob = p->desc;
  va.A = p->dA;
  va.lam = p->vlam.as<double2>();
  va.m = m;
  va.tol_verify = opt->tol_verify;
  va.sigma_min = p->vsig.as<double>();
  va.accept = p->vacc.as<uint8_t>();
  va.work = p->vwork.as<double2>();
  va.vec = p->vvec.as<double2>();
  va.piv = p->vpiv.as<int32_t>();
  va.slots = slots;
  prof_begin(PMCIM_K_VERIFY, s);
  CU(launch_verify_fp64(va, s));
  prof_end(PMCIM_K_VERIFY, s);
  CU(cudaMemcpyAsync(sig->data(), p->vsig.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(acc->data(), p->vacc.p, m, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

// Certificate sigma_min(T(lambda)) <= ||T(lambda) v|| for the gathered unit
// eigenvectors (p->gdst, same order as lam).
int run_certify(pmcim_problem p, const pmcim_options* opt, const std::vector<double2>& lam,
                std::vector<double>* cert, std::vector<uint8_t>* ok) {
  cudaStream_t s = stream_of(opt);
  const int m = (int)lam.size();
  cert->assign(m, 0.0);
  ok->assign(m, 0);
  if (m == 0) return PMCIM_OK;
  CU(p->vlam.ensure(m * sizeof(double2)));
  CU(p->vsig.ensure(m * sizeof(double)));
  CU(p->vacc.ensure(m));
  CU(cudaMemcpyAsync(p->vlam.p, lam.data(), m * sizeof(double2), cudaMemcpyHostToDevice, s));
  CertifyArgs ca;
  ca.prob = p->desc;
  ca.A = p->dA;
  ca.lam = p->vlam.as<double2>();
  ca.vecs = p->gdst.as<double2>();
  ca.m = m;
  ca.tol_verify = opt->tol_verify;
  ca.cert = p->vsig.as<double>();
  ca.certified = p->vacc.as<uint8_t>();
  prof_begin(PMCIM_K_VERIFY, s);
  CU(launch_certify(ca, s));
  prof_end(PMCIM_K_VERIFY, s);
  CU(cudaMemcpyAsync(cert->data(), p->vsig.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(ok->data(), p->vacc.p, m, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

std::vector<HostRegion> to_host_regions(int R, const pmcim_region* reg) {
  std::vector<HostRegion> v(R);
  for (int g = 0; g < R; ++g) v[g] = HostRegion{reg[g].c_re, reg[g].c_im, reg[g].r, reg[g].N, 0, g};
  return v;
}

int check_device() {
  int cnt = 0;
  cudaError_t e = cudaGetDeviceCount(&cnt);
  if (e != cudaSuccess || cnt == 0) return fail(PMCIM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  return PMCIM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void pmcim_default_options(pmcim_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->tol_ind = 0.1;
  opt->tol_svd = 1e-6;
  opt->tol_verify = 1e-6;
  opt->precision = PMCIM_PREC_FP64;
  opt->max_ir_sweeps = 3;
  opt->max_split_depth = 8;
  opt->cuda_stream = nullptr;
}

const char* pmcim_status_string(int code) {
  switch (code) {
    case PMCIM_OK: return "ok";
    case PMCIM_EINVAL: return "invalid argument";
    case PMCIM_ENOMEM: return "out of device memory";
    case PMCIM_ECUDA: return "CUDA error";
    case PMCIM_ETIMEOUT: return "device wait timed out";
    case PMCIM_ECAPACITY: return "output capacity exceeded";
    case PMCIM_ENOTSUP: return "not supported";
    default: return "unknown status";
  }
}

const char* pmcim_last_error(void) { return g_last_error.c_str(); }

void pmcim_profile_enable(int on) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.on = on != 0;
}

void pmcim_profile_reset(void) {
  prof_flush();
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  for (int k = 0; k < PMCIM_K_COUNT; ++k) {
    P.launches[k] = 0;
    P.ms[k] = 0.0;
  }
  for (int q = 0; q < 8; ++q) P.phase[q] = 0.0;
}

void pmcim_profile_read(pmcim_profile* out) {
  if (!out) return;
  prof_flush();
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  for (int k = 0; k < PMCIM_K_COUNT; ++k) {
    out->launches[k] = P.launches[k];
    out->ms[k] = P.ms[k];
  }
  for (int q = 0; q < 8; ++q) out->mixed_phase_cycles[q] = P.phase[q];
}

int pmcim_problem_create(int32_t n, int32_t K, const double* const* A, const pmcim_fterm* f, pmcim_problem* out) {
  if (!out) return fail(PMCIM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 16384) return fail(PMCIM_EINVAL, "n = %d outside 1..16384", n);
  if (K < 1 || K > PMCIM_MAX_TERMS) return fail(PMCIM_EINVAL, "K = %d outside 1..%d", K, PMCIM_MAX_TERMS);
  if (!A || !f) return fail(PMCIM_EINVAL, "A or f is NULL");
  CHK(check_device());
  pmcim_problem p = new pmcim_problem_s();
  p->n = n;
  p->K = K;
  p->desc.n = n;
  p->desc.K = K;
  int nd = 0;
  for (int k = 0; k < K; ++k) {
    if (f[k].kind != PMCIM_F_MONOMIAL && f[k].kind != PMCIM_F_EXP_NEG) {
      delete p;
      return fail(PMCIM_EINVAL, "term %d: unknown kind %d", k, f[k].kind);
    }
    if (f[k].kind == PMCIM_F_MONOMIAL && (f[k].degree < 0 || f[k].degree > 16)) {
      delete p;
      return fail(PMCIM_EINVAL, "term %d: degree %d outside 0..16", k, f[k].degree);
    }
    TermDesc& t = p->desc.term[k];
    t.kind = f[k].kind;
    t.degree = f[k].degree;
    t.tau = f[k].tau;
    t.id = make_double2(f[k].id_re, f[k].id_im);
    t.dense = A[k] ? 1 : 0;
    t.mat_index = A[k] ? nd++ : -1;
  }
  p->desc.n_dense = nd;
  cudaGetDevice(&p->device);
  const size_t nn = (size_t)n * n;
  if (nd > 0) {
    cudaError_t e = cudaMalloc(&p->dA, (size_t)nd * nn * sizeof(double2));
    if (e != cudaSuccess) {
      delete p;
      return fail(PMCIM_ENOMEM, "coefficient upload: %s", cudaGetErrorString(e));
    }
    for (int k = 0; k < K; ++k) {
      if (!A[k]) continue;
      e = cudaMemcpy(p->dA + (size_t)p->desc.term[k].mat_index * nn, A[k], nn * sizeof(double2), cudaMemcpyDefault);
      if (e != cudaSuccess) {
        cudaFree(p->dA);
        delete p;
        return fail(PMCIM_ECUDA, "coefficient upload: %s", cudaGetErrorString(e));
      }
    }
  }
  *out = p;
  return PMCIM_OK;
}

int pmcim_problem_destroy(pmcim_problem p) {
  if (!p) return PMCIM_OK;
  cudaDeviceSynchronize();
  if (p->dA) cudaFree(p->dA);
  DevBuf* bufs[] = {&p->work, &p->piv, &p->X, &p->node_info, &p->regions, &p->node_region, &p->V,
                    &p->C0, &p->C1, &p->pf_half, &p->pf_abs, &p->ind, &p->pf_norm, &p->pf_scale, &p->cand,
                    &p->bslot, &p->bregion, &p->bwork, &p->bsigma, &p->bp, &p->blam, &p->bvecs, &p->bkept,
                    &p->bstatus, &p->vlam, &p->vsig, &p->vacc, &p->vwork, &p->vvec, &p->vpiv, &p->gsrc, &p->gdst, &p->gperm, &p->phase};
  for (DevBuf* b : bufs) b->release();
  delete p;
  return PMCIM_OK;
}

int pmcim_moments(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
                  const double* V, double* C0, double* C1, double* pf_half, double* pf_abs) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l, p->n));
  cudaStream_t s = stream_of(opt);
  CHK(upload_V(p, l, V, s));
  std::vector<HostRegion> regs = to_host_regions(R, reg);
  CHK(run_moments(p, opt, regs, l, nullptr, nullptr));
  const size_t nl = (size_t)p->n * l;
  if (C0) CU(cudaMemcpyAsync(C0, p->C0.p, (size_t)R * nl * sizeof(double2), cudaMemcpyDefault, s));
  if (C1) CU(cudaMemcpyAsync(C1, p->C1.p, (size_t)R * nl * sizeof(double2), cudaMemcpyDefault, s));
  if (pf_half) CU(cudaMemcpyAsync(pf_half, p->pf_half.p, (size_t)R * p->n * sizeof(double2), cudaMemcpyDefault, s));
  if (pf_abs) CU(cudaMemcpyAsync(pf_abs, p->pf_abs.p, (size_t)R * p->n * sizeof(double), cudaMemcpyDefault, s));
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

int pmcim_indicator(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
                    const double* V, double* ind, double* pf_norm, double* pf_scale, uint8_t* candidate) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l, p->n));
  if (R > 0 && (!ind || !candidate)) return fail(PMCIM_EINVAL, "ind or candidate is NULL");
  cudaStream_t s = stream_of(opt);
  CHK(upload_V(p, l, V, s));
  std::vector<HostRegion> regs = to_host_regions(R, reg);
  CHK(run_moments(p, opt, regs, l, nullptr, nullptr));
  CHK(run_indicator(p, opt, R, l));
  if (R > 0) {
    CU(cudaMemcpyAsync(ind, p->ind.p, R * sizeof(double), cudaMemcpyDefault, s));
    CU(cudaMemcpyAsync(candidate, p->cand.p, R * sizeof(uint8_t), cudaMemcpyDefault, s));
    if (pf_norm) CU(cudaMemcpyAsync(pf_norm, p->pf_norm.p, R * sizeof(double), cudaMemcpyDefault, s));
    if (pf_scale) CU(cudaMemcpyAsync(pf_scale, p->pf_scale.p, R * sizeof(double), cudaMemcpyDefault, s));
  }
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

int pmcim_beyn(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
               const double* V, int32_t cap, double* lambda, double* vecs, int32_t* region_of, int32_t* count,
               int32_t* region_status) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l, p->n));
  if (!count || cap < 0 || (cap > 0 && !lambda)) return fail(PMCIM_EINVAL, "bad output arguments");
  cudaStream_t s = stream_of(opt);
  CHK(upload_V(p, l, V, s));
  EigOut out;
  std::vector<int> rstat;
  CHK(run_beyn_levels(p, opt, to_host_regions(R, reg), l, false, vecs != nullptr, &out, &rstat, nullptr,
                      nullptr));
  const int cnt = (int)out.lam.size();
  CHK(copy_out(count, &cnt, sizeof(int32_t)));
  if (region_status) CHK(copy_out(region_status, rstat.data(), R * sizeof(int32_t)));
  if (cnt > cap) return fail(PMCIM_ECAPACITY, "%d eigenvalues exceed capacity %d", cnt, cap);
  CHK(copy_out(lambda, out.lam.data(), cnt * sizeof(double2)));
  if (region_of) CHK(copy_out(region_of, out.root.data(), cnt * sizeof(int32_t)));
  if (vecs && cnt > 0) CHK(copy_out(vecs, p->gdst.p, (size_t)cnt * p->n * sizeof(double2)));
  return PMCIM_OK;
}

int pmcim_verify(pmcim_problem p, const pmcim_options* opt, int32_t m, const double* lambda, double* sigma_min,
                 uint8_t* accept) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  if (m < 0 || (m > 0 && (!lambda || !sigma_min))) return fail(PMCIM_EINVAL, "bad arguments");
  std::vector<double2> lam(m);
  if (m > 0) {
    cudaError_t e = cudaMemcpy(lam.data(), lambda, m * sizeof(double2), cudaMemcpyDefault);
    if (e != cudaSuccess) return fail(PMCIM_ECUDA, "lambda copy: %s", cudaGetErrorString(e));
  }
  std::vector<double> sig;
  std::vector<uint8_t> acc;
  CHK(run_verify(p, opt, lam, &sig, &acc));
  CHK(copy_out(sigma_min, sig.data(), m * sizeof(double)));
  if (accept) CHK(copy_out(accept, acc.data(), m));
  return PMCIM_OK;
}

int pmcim_solve(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
                const double* V, int32_t cap, double* lambda, double* vecs, double* sigma_min, int32_t* region_of,
                int32_t* count, double* ind, int32_t* region_status, pmcim_stats* stats) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l, p->n));
  if (!count || cap < 0 || (cap > 0 && !lambda)) return fail(PMCIM_EINVAL, "bad output arguments");
  cudaStream_t s = stream_of(opt);
  pmcim_stats st;
  std::memset(&st, 0, sizeof(st));
  CHK(upload_V(p, l, V, s));
  EigOut out;
  std::vector<int> rstat;
  std::vector<double> tind;
  const bool want_vecs = vecs != nullptr;
  // eigenvectors are always gathered: they carry the verification certificate
  CHK(run_beyn_levels(p, opt, to_host_regions(R, reg), l, true, true, &out, &rstat, &tind, &st));
  std::vector<double> sig;
  std::vector<uint8_t> acc;
  CHK(run_certify(p, opt, out.lam, &sig, &acc));
  {
    std::vector<double2> rest;
    std::vector<int> idx;
    for (size_t i = 0; i < out.lam.size(); ++i)
      if (acc[i]) st.certified += 1;
      else {
        rest.push_back(out.lam[i]);
        idx.push_back((int)i);
      }
    std::vector<double> sig2;
    std::vector<uint8_t> acc2;
    CHK(run_verify(p, opt, rest, &sig2, &acc2));
    for (size_t k = 0; k < idx.size(); ++k) {
      sig[idx[k]] = sig2[k];
      acc[idx[k]] = acc2[k];
    }
  }
  const int m = (int)out.lam.size();
  std::vector<int> order;
  for (int i = 0; i < m; ++i)
    if (acc[i]) order.push_back(i);
    else st.unverified += 1;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (out.lam[a].x != out.lam[b].x) return out.lam[a].x < out.lam[b].x;
    return out.lam[a].y < out.lam[b].y;
  });
  const int cnt = (int)order.size();
  CHK(copy_out(count, &cnt, sizeof(int32_t)));
  if (ind) CHK(copy_out(ind, tind.data(), R * sizeof(double)));
  if (region_status) CHK(copy_out(region_status, rstat.data(), R * sizeof(int32_t)));
  if (stats) CHK(copy_out(stats, &st, sizeof(st)));
  if (cnt > cap) return fail(PMCIM_ECAPACITY, "%d eigenvalues exceed capacity %d", cnt, cap);
  std::vector<double2> lam_s(cnt);
  std::vector<double> sig_s(cnt);
  std::vector<int32_t> root_s(cnt);
  for (int i = 0; i < cnt; ++i) {
    lam_s[i] = out.lam[order[i]];
    sig_s[i] = sig[order[i]];
    root_s[i] = out.root[order[i]];
  }
  CHK(copy_out(lambda, lam_s.data(), cnt * sizeof(double2)));
  if (sigma_min) CHK(copy_out(sigma_min, sig_s.data(), cnt * sizeof(double)));
  if (region_of) CHK(copy_out(region_of, root_s.data(), cnt * sizeof(int32_t)));
  if (want_vecs && cnt > 0) {
    // permute the gathered vectors into the sorted order on the device, one copy out
    std::vector<int32_t> src(order.begin(), order.end());
    CU(p->gsrc.ensure(cnt * sizeof(int32_t)));
    CU(p->gperm.ensure((size_t)cnt * p->n * sizeof(double2)));
    CU(cudaMemcpyAsync(p->gsrc.p, src.data(), cnt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    GatherArgs ga;
    ga.vecs = p->gdst.as<double2>();
    ga.src = p->gsrc.as<int32_t>();
    ga.dst = p->gperm.as<double2>();
    ga.n = p->n;
    ga.l = 1;
    ga.count = cnt;
    prof_begin(PMCIM_K_GATHER, s);
    CU(launch_gather_vecs(ga, s));
    prof_end(PMCIM_K_GATHER, s);
    CU(cudaStreamSynchronize(s));
    CHK(copy_out(vecs, p->gperm.p, (size_t)cnt * p->n * sizeof(double2)));
  }
  return PMCIM_OK;
}

}  // extern "C"
