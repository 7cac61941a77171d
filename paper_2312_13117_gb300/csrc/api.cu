// C ABI of libpmcim and the host-side control of pmCIMb (Sec. 3.2).
//
// The host side turns lists of disks (of one or many problems) into levels of
// work: every node of every disk of a level is one linear system. A level is
// captured as one CUDA graph: per HBM wave, the node kernels (one persistent
// launch per arithmetic form, work handed out largest-first) and the segmented
// reduction; then the indicator and Beyn's extraction over all disks of the
// level, gated on the device. The host reads the small per-disk results, splits
// saturated disks into four children (pmCIMa's quadrisection geometry, Sec.
// 3.1), and finally certifies or verifies the surviving values. All arithmetic
// of the method runs in the CUDA kernels; the host only builds work lists,
// moves small results and sorts.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
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

#define CU(expr)                                                                                  \
  do {                                                                                            \
    cudaError_t _e = (expr);                                                                      \
    if (_e != cudaSuccess)                                                                        \
      return fail(_e == cudaErrorMemoryAllocation ? PMCIM_ENOMEM : PMCIM_ECUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(_e), __FILE__, __LINE__);                             \
  } while (0)

#define CHK(expr)                  \
  do {                             \
    int _r = (expr);               \
    if (_r != PMCIM_OK) return _r; \
  } while (0)

// Growable device buffer.
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
      if (e != cudaSuccess) {
        cudaFree(q);
        return e;
      }
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
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

// Upper bound on the node solutions kept before one reduction (one HBM wave).
constexpr size_t kWaveBytes = size_t(16) << 30;
// Upper bound on the per-CTA factorisation workspaces of one form: at n = 2048 the
// precision form's 152 CTAs need 41 GB (two complex64 slots and two FP64 T(z_j) each).
constexpr size_t kSlotBytes = size_t(48) << 30;
// indicator-pass solutions kept for reuse by the two-pass schedule, per chunk of disks
constexpr size_t kKeepBytes = size_t(8) << 30;
// largest pmCIMa level (disks); beyond it the indicator is marking noise
constexpr size_t kMaxPmcimaRegions = size_t(1) << 20;
// Refinement stops when the estimated remaining error of X (max norm) is below
// this fraction of |X|: 1e-11 keeps Beyn's eigenvalues within about 1e-14 of
// the FP64 ones on the delay workload (simulated FP32 LU + FP64 refinement).
constexpr double kIrTol = 1e-11;
// Default limits of the precision-form kernel's bounded waits (clock64 cycles):
// a tensor-core commit (about half a second at 2 GHz) and a hand-off between its
// thread groups (about 16 s, longer than any node at n <= 4096).
constexpr long long kTcWaitCycles = 1ll << 30;
constexpr long long kHandoffWaitCycles = 1ll << 35;
std::mutex g_wait_mu;
long long g_tc_wait = kTcWaitCycles, g_handoff_wait = kHandoffWaitCycles;

// Bytes one form's factorisation workspaces may take now: at most kSlotBytes, and at
// most what they already hold plus 70 % of the device memory that is free, so that a
// GPU shared with other work gets fewer resident CTAs instead of a failed allocation.
size_t slot_budget(size_t held) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return kSlotBytes;
  return std::min(kSlotBytes, held + fr / 10 * 7);
}

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
  double phase[PMCIM_PHASE_COUNT] = {};
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

// A timing event. Inside stream capture a plain record only orders streams;
// the external flag makes it a real event-record node of the graph.
void record_timing_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
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
    for (int q = 0; q < PMCIM_PHASES; ++q) P.phase[q] += (double)c[(size_t)b * PMCIM_PHASES + q];
}

void prof_begin(int kind, cudaStream_t s) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.launches[kind] += 1;
  if (!P.on) return;
  cudaEvent_t e = P.get();
  record_timing_event(e, s);
  P.cur_begin[kind] = e;
}

void prof_end(int kind, cudaStream_t s) {
  Prof& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  if (!P.on || !P.cur_begin[kind]) return;
  cudaEvent_t e = P.get();
  record_timing_event(e, s);
  P.pending.push_back({kind, P.cur_begin[kind], e});
  P.cur_begin[kind] = nullptr;
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

long long wait_limit_tc() {
  std::lock_guard<std::mutex> g(g_wait_mu);
  return g_tc_wait;
}
long long wait_limit_handoff() {
  std::lock_guard<std::mutex> g(g_wait_mu);
  return g_handoff_wait;
}

// Device workspaces, reused across calls on one handle.
struct Workspace {
  DevBuf probs, regions, items, counters, node_info, X;
  DevBuf work64, piv64, work32, piv32, t64, phase;
  DevBuf C0, C1, pf_half, pf_abs, ind, pf_norm, pf_scale, cand;
  DevBuf bwork, bsigma, bp, blam, bvecs, bkept, bstatus;
  DevBuf vlam, vprob, voff, vsig, vacc, vwork, vvec, vpiv;
  DevBuf gitems, gdst, gperm;
  DevBuf Xkeep, citems;  // two-pass schedule: indicator-pass solutions, copy list
  DevBuf vout;           // verification's singular vectors (pmCIMa)
  DevBuf Cm;             // scaled moments of the block Hankel form of Beyn's step
  DevBuf ind3, feats, sprob, sparams, sscratch;
  // verification's inverse-iteration step: per-value problem table, pseudo-disks, items, solutions
  DevBuf iprobs, iregions, iitems, iX, iinfo, icounters, ibord, ioffs;
  DevBuf ysl;                        // per slot: digits of f_k X for the tensor-core residual
  DevBuf rz, rX, rR, rstat, rysl;    // pmcim_residual: points, solutions, residuals, status, scratch
  DevBuf cW, cidx, cgram, gpart;     // certificates from coefficient products: W, index arrays, Gram data
  // the library's own stream: graphs cannot be captured on the legacy default stream
  cudaStream_t stream = nullptr;
  cudaEvent_t ordered = nullptr;
  void release() {
    if (stream) cudaStreamDestroy(stream);
    if (ordered) cudaEventDestroy(ordered);
    stream = nullptr;
    ordered = nullptr;
    DevBuf* b[] = {&probs, &regions, &items, &counters, &node_info, &X, &work64, &piv64, &work32, &piv32, &t64,
                   &phase, &C0, &C1, &pf_half, &pf_abs, &ind, &pf_norm, &pf_scale, &cand, &bwork, &bsigma,
                   &bp, &blam, &bvecs, &bkept, &bstatus, &vlam, &vprob, &voff, &vsig, &vacc, &vwork,
                   &vvec, &vpiv, &gitems, &gdst, &gperm, &ind3, &feats, &sprob, &sparams, &sscratch, &Xkeep,
                   &citems, &vout, &Cm, &iprobs, &iregions, &iitems, &iX, &iinfo, &icounters, &ibord, &ioffs, &ysl, &rz,
                   &rX, &rR, &rstat, &rysl, &cW, &cidx, &cgram, &gpart};
    for (DevBuf* x : b) x->release();
  }
};

struct pmcim_problem_s {
  int n = 0, K = 0, n_dense = 0;
  TermDesc term[PMCIM_MAX_TERMS];
  double2* dA = nullptr;
  // geometry of the boundary-integral term (bie.cuh), NULL without one; such a
  // problem has no coefficient matrices for the precision forms and runs in FP64
  double* dG = nullptr;
  bool bie_circ = false;  // its matrix is circulant (bie.cuh)
  float2* dA32 = nullptr;  // complex64 copy for the FP32 LU's assembly
  // exact BF16 digits of the dense coefficients and their row exponents, made on
  // the first call that refines with residuals on the tensor cores
  DevBuf dig, dexp;
  bool dig_ok = false;
  // Gram data of the dense coefficients for the certificates (made on first use)
  DevBuf gram;
  bool gram_ok = false;
  int device = 0;
  DevBuf V;  // probe block of the current call
  Workspace ws;
};

namespace {

struct HostRegion {
  double cre, cim, r;
  int N;
  int depth;
  int root;  // index of the caller's disk this one descends from
  int prob;  // index of the problem (group) in the call
};

// Work of a call runs on the workspace's stream, ordered after everything the
// caller queued on opt->cuda_stream before the call.
int call_stream(Workspace& ws, const pmcim_options* opt, cudaStream_t* out) {
  if (!ws.stream) CU(cudaStreamCreateWithFlags(&ws.stream, cudaStreamNonBlocking));
  if (!ws.ordered) CU(cudaEventCreateWithFlags(&ws.ordered, cudaEventDisableTiming));
  CU(cudaEventRecord(ws.ordered, reinterpret_cast<cudaStream_t>(opt->cuda_stream)));
  CU(cudaStreamWaitEvent(ws.stream, ws.ordered, 0));
  *out = ws.stream;
  return PMCIM_OK;
}

// One problem of a call: handle, probe count, arithmetic form.
struct Group {
  pmcim_problem h;
  int l;
  int form;       // PMCIM_PREC_FP64, PMCIM_PREC_FP32_IR, PMCIM_PREC_TF32X3_IR or PMCIM_PREC_BF16X3_IR
  int tile = 64;  // FP64 form: trailing-update tile of the node kernel (32 or 64)
};

// whether any problem of the call has a boundary-integral term (selects the kernel
// instantiations that assemble its entries)
bool any_bie(const std::vector<Group>& groups) {
  for (const Group& g : groups)
    if (g.h->dG) return true;
  return false;
}

int check_options(const pmcim_options* opt) {
  if (!opt) return fail(PMCIM_EINVAL, "options pointer is NULL");
  if (!(opt->tol_ind >= 0.0) || !(opt->tol_svd >= 0.0) || !(opt->tol_verify >= 0.0))
    return fail(PMCIM_EINVAL, "tolerances must be non-negative");
  if (opt->precision != PMCIM_PREC_FP64 && opt->precision != PMCIM_PREC_FP32_IR &&
      opt->precision != PMCIM_PREC_AUTO && opt->precision != PMCIM_PREC_TF32X3_IR &&
      opt->precision != PMCIM_PREC_BF16X3_IR)
    return fail(PMCIM_EINVAL, "unknown precision %d", opt->precision);
  if (opt->max_split_depth < 0 || opt->max_split_depth > 30) return fail(PMCIM_EINVAL, "max_split_depth out of range");
  if (opt->precision != PMCIM_PREC_FP64 && (opt->max_ir_sweeps < 1 || opt->max_ir_sweeps > 10))
    return fail(PMCIM_EINVAL, "max_ir_sweeps must be 1..10");
  if (opt->tol_ir != 0.0 && !(opt->tol_ir >= 1e-15 && opt->tol_ir <= 1e-6))
    return fail(PMCIM_EINVAL, "tol_ir must be 0 (default) or in [1e-15, 1e-6]");
  if (opt->indicator_N != 0 && (opt->indicator_N < 2 || opt->indicator_N > 4096 || (opt->indicator_N & 1)))
    return fail(PMCIM_EINVAL, "indicator_N = %d must be 0 or even, 2..4096", opt->indicator_N);
  if (opt->residual_fp64 != 0 && opt->residual_fp64 != 1)
    return fail(PMCIM_EINVAL, "residual_fp64 = %d must be 0 or 1", opt->residual_fp64);
  if (opt->fp64_tile != 0 && opt->fp64_tile != 32 && opt->fp64_tile != 64)
    return fail(PMCIM_EINVAL, "fp64_tile = %d must be 0, 32 or 64", opt->fp64_tile);
  if (opt->beyn_K < 0 || opt->beyn_K > PMCIM_MAX_BEYN_K)
    return fail(PMCIM_EINVAL, "beyn_K = %d outside 0..%d", opt->beyn_K, PMCIM_MAX_BEYN_K);
  return PMCIM_OK;
}

int check_regions(int R, const pmcim_region* reg, int l) {
  if (R < 0) return fail(PMCIM_EINVAL, "negative region count");
  if (R > 0 && !reg) return fail(PMCIM_EINVAL, "regions pointer is NULL");
  if (l < 1 || l > PMCIM_MAX_L) return fail(PMCIM_EINVAL, "l = %d outside 1..%d", l, PMCIM_MAX_L);
  for (int g = 0; g < R; ++g) {
    if (reg[g].N < 2 || reg[g].N > 4096 || (reg[g].N & 1))
      return fail(PMCIM_EINVAL, "region %d: N = %d must be even, 2..4096", g, reg[g].N);
    if (!(reg[g].r > 0.0) || !std::isfinite(reg[g].r) || !std::isfinite(reg[g].c_re) || !std::isfinite(reg[g].c_im))
      return fail(PMCIM_EINVAL, "region %d: bad centre or radius", g);
  }
  return PMCIM_OK;
}

int upload_V(pmcim_problem p, int l, const double* V, cudaStream_t s) {
  if (!V) return fail(PMCIM_EINVAL, "V is NULL");
  const size_t bytes = (size_t)p->n * l * sizeof(double2);
  CU(p->V.ensure(bytes));
  CU(cudaMemcpyAsync(p->V.p, V, bytes, cudaMemcpyDefault, s));
  return PMCIM_OK;
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// ===========================================================================
// One call's view of its problems
// ===========================================================================
struct Call {
  const pmcim_options* opt;
  cudaStream_t s;
  Workspace* ws;
  std::vector<Group> groups;
  std::vector<ProblemDev> pd;  // host copy of the device problem table
  pmcim_stats st{};
  int tile_override = 0;       // autotuner probes: the FP64 kernel's tile (0: the groups')
};

// The coefficient digits of a handle for the tensor-core residuals (ozaki.cuh),
// made once; ordered before later work on stream s.
int ensure_digits(pmcim_problem h, cudaStream_t s) {
  if (h->dig_ok || h->n_dense == 0) return PMCIM_OK;
  const int RB = (h->n + 127) / 128;
  CU(h->dexp.ensure((size_t)h->n_dense * RB * 128 * sizeof(int32_t)));
  CU(h->dig.ensure(coefficient_digit_bytes(h->n, h->n_dense)));
  CU(make_coefficient_digits(h->dA, h->n, h->n_dense, h->dexp.as<int32_t>(), h->dig.as<unsigned char>(), s));
  h->dig_ok = true;
  return PMCIM_OK;
}

// Residuals of the precision forms on the tensor cores (default) or the FP64 pipe.
bool tc_residual(const pmcim_options* opt) { return opt->residual_fp64 == 0; }

int upload_problems(Call& c) {
  if (c.opt->precision != PMCIM_PREC_FP64 && tc_residual(c.opt))
    for (const Group& g : c.groups) CHK(ensure_digits(g.h, c.s));
  c.pd.resize(c.groups.size());
  for (size_t i = 0; i < c.groups.size(); ++i) {
    const Group& g = c.groups[i];
    ProblemDev& d = c.pd[i];
    std::memset(&d, 0, sizeof(d));
    d.n = g.h->n;
    d.K = g.h->K;
    d.l = g.l;
    d.n_dense = g.h->n_dense;
    d.A = g.h->dA;
    d.A32 = g.h->dA32;
    d.Adig = g.h->dig_ok ? g.h->dig.as<unsigned char>() : nullptr;
    d.Aexp = g.h->dig_ok ? g.h->dexp.as<int32_t>() : nullptr;
    d.bie = g.h->dG;
    d.bie_circ = g.h->bie_circ ? 1 : 0;
    d.V = g.h->V.as<double2>();
    for (int k = 0; k < g.h->K; ++k) d.term[k] = g.h->term[k];
  }
  CU(c.ws->probs.ensure(std::max<size_t>(1, c.pd.size()) * sizeof(ProblemDev)));
  CU(cudaMemcpyAsync(c.ws->probs.p, c.pd.data(), c.pd.size() * sizeof(ProblemDev), cudaMemcpyHostToDevice, c.s));
  return PMCIM_OK;
}

// ===========================================================================
// Autotuner: per (n-bucket, l, dense terms), FP64 or one of the two precision
// forms, whichever solves nodes fastest on this device (measured once per
// process).
// ===========================================================================
struct TuneKey {
  int bucket, l, kd;
  bool operator<(const TuneKey& o) const { return std::tie(bucket, l, kd) < std::tie(o.bucket, o.l, o.kd); }
};
std::mutex g_tune_mu;
struct TuneChoice {
  int form, tile;
};
std::map<TuneKey, TuneChoice> g_tune;
// FP64 node kernels with 32 x 32 trailing tiles are tried up to this n
constexpr int kTile32MaxN = 256;

int n_bucket(int n) {
  int b = 0;
  while ((32 << b) < n) ++b;  // buckets (..32], (32,64], (64,128], ...
  return b;
}

struct LevelOut {
  std::vector<double> ind;
  std::vector<uint8_t> cand;
  std::vector<int32_t> p, status, node_info;
  std::vector<double2> lam;
  std::vector<uint8_t> kept;
  std::vector<RegionDev> rd;
};

// Node solutions a level takes over from an earlier pass instead of solving
// them: for region g with src[g] >= 0, node j = m * stride[g] (m = 0, 1, ...)
// is copied from X + src[g] + m n l.
struct LevelReuse {
  const double2* X = nullptr;
  std::vector<int64_t> src;
  std::vector<int> stride;
};

// gate_top: the indicator gates Beyn for depth-0 disks too (deeper ones always);
// no_gate: Beyn runs on every disk; keep_x: all solutions of the level stay in
// ws.Xkeep (one wave), at rd[g].x_off, for a later pass to reuse.
int run_level(Call& c, const std::vector<HostRegion>& regs, bool gate_top, bool do_beyn, LevelOut* out,
              const std::vector<int>* form_override = nullptr, bool screen_features = false,
              const LevelReuse* reuse = nullptr, bool keep_x = false, bool no_gate = false);

int tune_forms(Call& c) {
  if (c.opt->precision != PMCIM_PREC_AUTO) {
    for (Group& g : c.groups) {
      g.form = c.opt->precision;
      g.tile = c.opt->fp64_tile ? c.opt->fp64_tile : 64;
    }
    return PMCIM_OK;
  }
  for (size_t gi = 0; gi < c.groups.size(); ++gi) {
    Group& g = c.groups[gi];
    if (g.h->dG) {
      // A boundary-integral term is not timed on the probe's far-out disk: there its
      // entries grow like e^{|Im z| r} and its matrix would overflow FP32. The FP32 LU with
      // FP64 refinement is taken instead, the fastest form measured on the scattering-pole
      // workload (n = 256: 3.4 times plain FP64).
      g.form = PMCIM_PREC_FP32_IR;
      g.tile = c.opt->fp64_tile ? c.opt->fp64_tile : 64;
      c.st.tuned_mixed += 1;
      continue;
    }
    const TuneKey key{n_bucket(g.h->n), g.l, g.h->n_dense};
    TuneChoice decided{-1, 64};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) decided = it->second;
    }
    if (decided.form < 0) {
      // probe: one disk of 2 x SMs nodes on this problem, every candidate, timed with
      // events. It measures arithmetic throughput, so it sits far out (|z| ~ 70),
      // where the leading term dominates T(z) and no node is near an eigenvalue;
      // nodes next to eigenvalues would send the precision form to its FP64
      // fallback and misrepresent it. Candidates: FP64 with 64 x 64 trailing tiles,
      // FP64 with 32 x 32 tiles (small n only), and the two precision forms.
      std::vector<HostRegion> probe(1);
      probe[0] = HostRegion{50.0, 50.0, 1.0, 2 * num_sms(), 0, 0, (int)gi};
      // each candidate runs once untimed (workspace allocation, first launch), then timed
      const TuneChoice cands[5] = {{PMCIM_PREC_FP64, 64}, {PMCIM_PREC_FP64, 32}, {PMCIM_PREC_FP32_IR, 64},
                                   {PMCIM_PREC_TF32X3_IR, 64}, {PMCIM_PREC_BF16X3_IR, 64}};
      double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      const pmcim_stats keep = c.st;
      int best = -1;
      for (int f = 0; f < 5; ++f) {
        if (cands[f].tile == 32 && g.h->n > kTile32MaxN) continue;
        std::vector<int> ov(c.groups.size(), cands[f].form);
        c.tile_override = cands[f].tile;
        cudaEvent_t a, b;
        CU(cudaEventCreate(&a));
        CU(cudaEventCreate(&b));
        LevelOut lo;
        CHK(run_level(c, probe, false, false, &lo, &ov));
        CU(cudaEventRecord(a, c.s));
        CHK(run_level(c, probe, false, false, &lo, &ov));
        CU(cudaEventRecord(b, c.s));
        CU(cudaEventSynchronize(b));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, a, b));
        t[f] = ms;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (best < 0 || t[f] < t[best]) best = f;
      }
      c.tile_override = 0;
      c.st = keep;  // probe work is not part of the call's statistics
      decided = cands[best];
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = decided;
    }
    g.form = decided.form;
    g.tile = c.opt->fp64_tile ? c.opt->fp64_tile : decided.tile;
    if (decided.form == PMCIM_PREC_FP64) c.st.tuned_fp64 += 1;
    else if (decided.form == PMCIM_PREC_FP32_IR) c.st.tuned_mixed += 1;
    else c.st.tuned_tc += 1;
  }
  return PMCIM_OK;
}

// ===========================================================================
// One level: node solves (waves), reduction, indicator, Beyn (gated)
// ===========================================================================
int run_level(Call& c, const std::vector<HostRegion>& regs, bool gate_top, bool do_beyn, LevelOut* out,
              const std::vector<int>* form_override, bool screen_features, const LevelReuse* reuse, bool keep_x,
              bool no_gate) {
  Workspace& ws = *c.ws;
  cudaStream_t s = c.s;
  const int R = (int)regs.size();
  out->rd.assign(R, RegionDev{});
  if (R == 0) return PMCIM_OK;
  auto form_of = [&](int prob) { return form_override ? (*form_override)[prob] : c.groups[prob].form; };

  // ---- offsets of every disk's blocks ----
  // K > 1: Beyn on the block Hankel matrices of 2K scaled moments (K l columns)
  const int K = do_beyn ? std::max(1, c.opt->beyn_K) : 1;
  int max_n = 0, max_l = 0, max_nl = 0;
  size_t c_tot = 0, p_tot = 0, w_tot = 0, v_tot = 0, total_nodes = 0;
  std::vector<RegionDev>& rd = out->rd;
  for (int g = 0; g < R; ++g) {
    const HostRegion& h = regs[g];
    const ProblemDev& P = c.pd[h.prob];
    RegionDev& d = rd[g];
    d.cre = h.cre;
    d.cim = h.cim;
    d.r = h.r;
    d.N = h.N;
    d.prob = h.prob;
    d.node_off = (int32_t)total_nodes;
    d.gate = no_gate ? 0 : ((h.depth > 0 || gate_top) ? 1 : 0);
    d.lu_tc = form_of(h.prob) == PMCIM_PREC_TF32X3_IR ? 1 : form_of(h.prob) == PMCIM_PREC_BF16X3_IR ? 2 : 0;
    d.c_off = (int64_t)c_tot;
    d.p_off = (int64_t)p_tot;
    d.w_off = (int64_t)w_tot;
    d.v_off = (int64_t)v_tot;
    if (K * P.l > PMCIM_MAX_L)
      return fail(PMCIM_EINVAL, "beyn_K = %d with l = %d exceeds %d Beyn columns", K, P.l, PMCIM_MAX_L);
    const size_t rows = (size_t)K * P.n, cols = (size_t)K * P.l;
    c_tot += (size_t)P.n * P.l;
    p_tot += (size_t)P.n;
    v_tot += (size_t)P.n * cols;
    w_tot += (K == 1 ? 2 : 3) * rows * cols + 4 * cols * cols;
    total_nodes += (size_t)h.N;
    max_n = std::max(max_n, P.n);
    max_l = std::max(max_l, P.l);
    max_nl = std::max(max_nl, P.n * P.l);
  }
  CU(ws.C0.ensure(c_tot * sizeof(double2)));
  CU(ws.C1.ensure(c_tot * sizeof(double2)));
  CU(ws.pf_half.ensure(p_tot * sizeof(double2)));
  CU(ws.pf_abs.ensure(p_tot * sizeof(double)));
  CU(ws.ind.ensure(R * sizeof(double)));
  CU(ws.pf_norm.ensure(R * sizeof(double)));
  CU(ws.pf_scale.ensure(R * sizeof(double)));
  CU(ws.cand.ensure(R));
  CU(ws.node_info.ensure(std::max<size_t>(1, total_nodes) * sizeof(int32_t)));
  if (screen_features) {
    CU(ws.ind3.ensure((size_t)R * 3 * sizeof(double)));
    CU(ws.feats.ensure((size_t)R * 3 * sizeof(float)));
  }
  if (do_beyn) {
    CU(ws.bwork.ensure(w_tot * sizeof(double2)));
    CU(ws.bvecs.ensure(v_tot * sizeof(double2)));
    if (K > 1) CU(ws.Cm.ensure((size_t)2 * K * c_tot * sizeof(double2)));
    CU(ws.bsigma.ensure((size_t)R * PMCIM_MAX_L * sizeof(double)));
    CU(ws.blam.ensure((size_t)R * PMCIM_MAX_L * sizeof(double2)));
    CU(ws.bkept.ensure((size_t)R * PMCIM_MAX_L));
    CU(ws.bp.ensure(R * sizeof(int32_t)));
    CU(ws.bstatus.ensure(R * sizeof(int32_t)));
  }

  // ---- waves of whole disks whose solutions fit the wave buffer ----
  struct Wave {
    int g0, g1;
    size_t items64_off, n64, items32_off, n32, itemsS_off, nS;
    size_t copies_off, n_copies;  // reused solutions copied into this wave's X
    int max_copy;
  };
  std::vector<Wave> waves;
  std::vector<NodeItem> items;  // all waves: FP64 items then mixed items per wave
  std::vector<VecItem> copies;  // all waves
  size_t x_need = 0, reused_nodes = 0;
  bool any64 = false, any32 = false, anyS = false;
  int t64_n = 0;  // largest n of a precision-form problem with two or more dense terms
  int ysl_n = 0, ysl_nd = 0;  // largest n and dense-term count of the tensor-core residuals
  {
    int g0 = 0;
    while (g0 < R) {
      int g1 = g0;
      size_t xb = 0;
      while (g1 < R && g1 - g0 < 65535) {
        const ProblemDev& P = c.pd[regs[g1].prob];
        const size_t b = (size_t)regs[g1].N * P.n * P.l * sizeof(double2);
        if (g1 > g0 && xb + b > kWaveBytes && !keep_x) break;
        rd[g1].x_off = (int64_t)(xb / sizeof(double2));
        xb += b;
        ++g1;
      }
      x_need = std::max(x_need, xb);
      // largest n first: the atomic work counter then hands out the long jobs early
      // small problems (n <= 32, l <= 16) go to the warp-per-node kernel whatever the form
      std::vector<NodeItem> it64, it32, itS;
      const size_t copies_off = copies.size();
      int max_copy = 0;
      for (int g = g0; g < g1; ++g) {
        const ProblemDev& P = c.pd[regs[g].prob];
        std::vector<NodeItem>& dst = small_kernel_fits(P.n, P.l) ? itS
                                     : (form_of(regs[g].prob) == PMCIM_PREC_FP64 ? it64 : it32);
        if (&dst == &it32 && ((P.n_dense >= 2 && !tc_residual(c.opt)) || P.bie)) t64_n = std::max(t64_n, P.n);
        if (&dst == &it32 && tc_residual(c.opt)) {
          ysl_n = std::max(ysl_n, P.n);
          ysl_nd = std::max(ysl_nd, P.n_dense);
        }
        const bool re = reuse && reuse->src[g] >= 0;
        const int nl = P.n * P.l;
        for (int j = 0; j < regs[g].N; ++j) {
          if (re && j % reuse->stride[g] == 0) {
            copies.push_back(VecItem{reuse->src[g] + (int64_t)(j / reuse->stride[g]) * nl,
                                     rd[g].x_off + (int64_t)j * nl, nl, 0});
            max_copy = std::max(max_copy, nl);
            ++reused_nodes;
          } else {
            dst.push_back(NodeItem{g, j});
          }
        }
      }
      auto by_n = [&](const NodeItem& a, const NodeItem& b) {
        const int na = c.pd[regs[a.region].prob].n, nb = c.pd[regs[b.region].prob].n;
        if (na != nb) return na > nb;
        if (a.region != b.region) return a.region < b.region;
        return a.j < b.j;
      };
      std::stable_sort(it64.begin(), it64.end(), by_n);
      std::stable_sort(it32.begin(), it32.end(), by_n);
      Wave wv{g0, g1, items.size(), it64.size(), 0, it32.size(), 0, itS.size(), copies_off,
              copies.size() - copies_off, max_copy};
      items.insert(items.end(), it64.begin(), it64.end());
      wv.items32_off = items.size();
      items.insert(items.end(), it32.begin(), it32.end());
      wv.itemsS_off = items.size();
      items.insert(items.end(), itS.begin(), itS.end());
      any64 |= !it64.empty();
      any32 |= !it32.empty();
      anyS |= !itS.empty();
      waves.push_back(wv);
      g0 = g1;
    }
  }
  DevBuf& xbuf = keep_x ? ws.Xkeep : ws.X;
  CU(xbuf.ensure(std::max<size_t>(1, x_need)));
  if (!copies.empty()) {
    CU(ws.citems.ensure(copies.size() * sizeof(VecItem)));
    CU(cudaMemcpyAsync(ws.citems.p, copies.data(), copies.size() * sizeof(VecItem), cudaMemcpyHostToDevice, s));
  }
  CU(ws.items.ensure(std::max<size_t>(1, items.size()) * sizeof(NodeItem)));
  CU(ws.regions.ensure(R * sizeof(RegionDev)));
  // 3 work counters per wave, then the mixed kernel's error flag
  CU(ws.counters.ensure((3 * waves.size() + 1) * sizeof(int)));
  CU(cudaMemcpyAsync(ws.items.p, items.data(), items.size() * sizeof(NodeItem), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ws.regions.p, rd.data(), R * sizeof(RegionDev), cudaMemcpyHostToDevice, s));

  // the FP64 kernel's trailing tile: 32 when every FP64-form problem of the level was
  // tuned to it (or an autotuner probe asks for it), else 64
  int fp64_tile = c.tile_override;
  if (!fp64_tile) {
    bool any = false, all32 = true;
    for (int g = 0; g < R; ++g)
      if (form_of(regs[g].prob) == PMCIM_PREC_FP64) {
        any = true;
        all32 = all32 && c.groups[regs[g].prob].tile == 32;
      }
    fp64_tile = (any && all32) ? 32 : 64;
  }
  // ---- factorisation workspaces, one slot per resident CTA ----
  const int sms = num_sms();
  int slots64 = 0, slots32 = 0;
  size_t slot64 = 0, slot32 = 0, t64_stride = 0, ysl_stride = 0;
  if (any64) {
    slot64 = (size_t)max_n * (max_n + max_l) * sizeof(double2);
    const size_t budget = slot_budget(ws.work64.cap);
    slots64 = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>(2 * sms, budget / slot64), total_nodes));
    CU(ws.work64.ensure((size_t)slots64 * slot64));
    CU(ws.piv64.ensure((size_t)slots64 * max_n * sizeof(int32_t)));
  }
  if (any32) {
    // one CTA per SM, each cycling through mixed_slots_per_cta() slots
    slot32 = mixed_slot_bytes(max_n, max_l);
    const size_t per = (size_t)mixed_slots_per_cta();
    t64_stride = (size_t)t64_n * t64_n;  // FP64 T(z_j) of each slot
    ysl_stride = y_digit_scratch_bytes(ysl_n, ysl_nd);
    const size_t cta_bytes = per * (slot32 + t64_stride * sizeof(double2) + ysl_stride);
    const size_t budget = slot_budget(ws.work32.cap + ws.t64.cap + ws.ysl.cap);
    const size_t ctas = std::max<size_t>(1, std::min<size_t>(std::min<size_t>(sms, budget / cta_bytes),
                                                             total_nodes));
    slots32 = (int)(ctas * per);
    c.st.node_ctas = std::max(c.st.node_ctas, (int32_t)ctas);
    CU(ws.work32.ensure((size_t)slots32 * slot32));
    CU(ws.piv32.ensure((size_t)slots32 * max_n * sizeof(int32_t)));
    if (t64_stride) CU(ws.t64.ensure((size_t)slots32 * t64_stride * sizeof(double2)));
    if (ysl_stride) CU(ws.ysl.ensure((size_t)slots32 * ysl_stride));
  }
  const bool timed = prof_on();
  if (timed && any32) {
    CU(ws.phase.ensure((size_t)slots32 * PMCIM_PHASES * sizeof(unsigned long long)));
    CU(cudaMemsetAsync(ws.phase.p, 0, (size_t)slots32 * PMCIM_PHASES * sizeof(unsigned long long), s));
  }

  LevelArgs la;
  std::memset(&la, 0, sizeof(la));
  la.probs = ws.probs.as<ProblemDev>();
  la.regions = ws.regions.as<RegionDev>();
  la.R = R;
  la.max_nl = max_nl;
  la.X = xbuf.as<double2>();
  la.C0 = ws.C0.as<double2>();
  la.C1 = ws.C1.as<double2>();
  la.K = K;
  la.Cm = K > 1 ? ws.Cm.as<double2>() : nullptr;
  la.pf_half = ws.pf_half.as<double2>();
  la.pf_abs = ws.pf_abs.as<double>();
  la.tol_ind = c.opt->tol_ind;
  la.tol_svd = c.opt->tol_svd;
  la.ind = ws.ind.as<double>();
  la.pf_norm = ws.pf_norm.as<double>();
  la.pf_scale = ws.pf_scale.as<double>();
  la.cand = ws.cand.as<uint8_t>();
  la.bwork = ws.bwork.as<double2>();
  la.sigma = ws.bsigma.as<double>();
  la.p = ws.bp.as<int32_t>();
  la.lam = ws.blam.as<double2>();
  la.vecs = ws.bvecs.as<double2>();
  la.kept = ws.bkept.as<uint8_t>();
  la.status = ws.bstatus.as<int32_t>();

  if (any64) CU(prepare_factor_fp64());
  if (any32) CU(prepare_factor_mixed());
  if (anyS) CU(prepare_factor_small());

  // ---- the level as one CUDA graph (profiler events become graph nodes) ----
  cudaGraph_t graph = nullptr;
  CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  auto capture = [&]() -> int {
    CU(cudaMemsetAsync(ws.counters.p, 0, (3 * waves.size() + 1) * sizeof(int), s));
    for (size_t wi = 0; wi < waves.size(); ++wi) {
      const Wave& wv = waves[wi];
      NodeArgs na;
      std::memset(&na, 0, sizeof(na));
      na.bie = any_bie(c.groups) ? 1 : 0;
      na.probs = la.probs;
      na.regions = la.regions;
      na.X = xbuf.as<double2>();
      // solutions taken over from an earlier pass
      for (size_t q0 = 0; q0 < wv.n_copies; q0 += 65535) {
        const int cnt = (int)std::min<size_t>(65535, wv.n_copies - q0);
        prof_begin(PMCIM_K_GATHER, s);
        CU(launch_gather_vecs(reuse->X, xbuf.as<double2>(), ws.citems.as<VecItem>() + wv.copies_off + q0, cnt,
                              wv.max_copy, s));
        prof_end(PMCIM_K_GATHER, s);
      }
      na.node_info = ws.node_info.as<int32_t>();
      na.max_n = max_n;
      na.max_sweeps = c.opt->max_ir_sweeps;
      na.tol_ir = c.opt->tol_ir > 0.0 ? c.opt->tol_ir : kIrTol;
      na.err = ws.counters.as<int32_t>() + 3 * waves.size();
      na.tc_wait_cycles = wait_limit_tc();
      na.handoff_wait_cycles = wait_limit_handoff();
      if (wv.n64) {
        na.items = ws.items.as<NodeItem>() + wv.items64_off;
        na.n_items = (int)wv.n64;
        na.fp64_tile = fp64_tile;
        na.counter = ws.counters.as<int>() + 3 * wi;
        na.work = ws.work64.as<char>();
        na.slot_bytes = slot64;
        na.piv = ws.piv64.as<int32_t>();
        na.slots = slots64;
        na.phase = nullptr;
        prof_begin(PMCIM_K_FACTOR, s);
        CU(launch_factor_solve_fp64(na, s));
        prof_end(PMCIM_K_FACTOR, s);
      }
      if (wv.n32) {
        na.items = ws.items.as<NodeItem>() + wv.items32_off;
        na.n_items = (int)wv.n32;
        na.counter = ws.counters.as<int>() + 3 * wi + 1;
        na.work = ws.work32.as<char>();
        na.slot_bytes = slot32;
        na.piv = ws.piv32.as<int32_t>();
        na.slots = slots32;
        na.t64 = t64_stride ? ws.t64.as<double2>() : nullptr;
        na.t64_stride = t64_stride;
        na.oz = tc_residual(c.opt) ? 1 : 0;
        na.ysl = ysl_stride ? ws.ysl.as<unsigned char>() : nullptr;
        na.ysl_stride = ysl_stride;
        na.phase = timed ? ws.phase.as<unsigned long long>() : nullptr;
        prof_begin(PMCIM_K_FACTOR32, s);
        CU(launch_factor_solve_mixed(na, s));
        prof_end(PMCIM_K_FACTOR32, s);
      }
      if (wv.nS) {
        na.items = ws.items.as<NodeItem>() + wv.itemsS_off;
        na.n_items = (int)wv.nS;
        na.counter = ws.counters.as<int>() + 3 * wi + 2;
        na.phase = nullptr;
        prof_begin(PMCIM_K_FACTOR, s);
        CU(launch_factor_solve_small(na, s));
        prof_end(PMCIM_K_FACTOR, s);
      }
      LevelArgs lw = la;
      lw.regions = la.regions + wv.g0;
      lw.R = wv.g1 - wv.g0;
      if (screen_features) {
        prof_begin(PMCIM_K_INDICATOR, s);
        CU(launch_screen_features(lw, ws.ind3.as<double>() + 3 * (size_t)wv.g0, s));
        prof_end(PMCIM_K_INDICATOR, s);
        continue;
      }
      prof_begin(PMCIM_K_REDUCE, s);
      CU(launch_reduce_moments(lw, s));
      prof_end(PMCIM_K_REDUCE, s);
    }
    if (screen_features) {
      CU(launch_make_features(R, ws.ind3.as<double>(), la.regions, ws.feats.as<float>(), s));
      return PMCIM_OK;
    }
    prof_begin(PMCIM_K_INDICATOR, s);
    CU(launch_indicator(la, s));
    prof_end(PMCIM_K_INDICATOR, s);
    if (do_beyn) {
      prof_begin(PMCIM_K_BEYN, s);
      CU(launch_beyn(la, s));
      prof_end(PMCIM_K_BEYN, s);
    }
    return PMCIM_OK;
  };
  const int cap_err = capture();
  cudaError_t ee = cudaStreamEndCapture(s, &graph);
  if (cap_err != PMCIM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return cap_err;
  }
  CU(ee);
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CU(ie);
  cudaError_t le = cudaGraphLaunch(exec, s);
  if (le == cudaSuccess) le = cudaStreamSynchronize(s);
  cudaGraphExecDestroy(exec);
  CU(le);
  c.st.graphs += 1;

  // ---- small per-disk results back to the host ----
  out->ind.resize(R);
  out->cand.resize(R);
  out->node_info.resize(total_nodes);
  if (!screen_features) {
    CU(cudaMemcpyAsync(out->ind.data(), ws.ind.p, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(out->cand.data(), ws.cand.p, R, cudaMemcpyDeviceToHost, s));
  }
  CU(cudaMemcpyAsync(out->node_info.data(), ws.node_info.p, total_nodes * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  int32_t handoff_err = 0;
  CU(cudaMemcpyAsync(&handoff_err, ws.counters.as<int32_t>() + 3 * waves.size(), sizeof(int32_t),
                     cudaMemcpyDeviceToHost, s));
  if (do_beyn) {
    out->p.resize(R);
    out->status.resize(R);
    out->lam.resize((size_t)R * PMCIM_MAX_L);
    out->kept.resize((size_t)R * PMCIM_MAX_L);
    CU(cudaMemcpyAsync(out->p.data(), ws.bp.p, R * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(out->status.data(), ws.bstatus.p, R * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(out->lam.data(), ws.blam.p, (size_t)R * PMCIM_MAX_L * sizeof(double2), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(out->kept.data(), ws.bkept.p, (size_t)R * PMCIM_MAX_L, cudaMemcpyDeviceToHost, s));
  }
  if (timed && any32) {
    std::vector<unsigned long long> cyc((size_t)slots32 * PMCIM_PHASES);
    CU(cudaMemcpyAsync(cyc.data(), ws.phase.p, cyc.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    prof_add_phases(cyc.data(), slots32);
  }
  CU(cudaStreamSynchronize(s));
  if (handoff_err)
    return fail(PMCIM_ETIMEOUT, "precision-form node kernel: a wait between its thread groups ran out");
  if (reuse)  // reused nodes were not solved here: their info words are stale
    for (int g = 0; g < R; ++g)
      if (reuse->src[g] >= 0)
        for (int j = 0; j < regs[g].N; j += reuse->stride[g]) out->node_info[rd[g].node_off + j] = 0;
  c.st.solves += (int64_t)(total_nodes - reused_nodes);
  int recount = 0;  // disks already counted by the pass their solutions come from
  if (reuse)
    for (int g = 0; g < R; ++g) recount += reuse->src[g] >= 0 ? 1 : 0;
  c.st.regions += R - recount;
  for (size_t i = 0; i < total_nodes; ++i) {
    const int v = out->node_info[i];
    if (v & (1 << 30)) c.st.ir_fallbacks += 1;
    if (v & (1 << 29)) c.st.tc_timeouts += 1;
    c.st.ir_sweeps += (v >> 24) & 31;
  }
  return PMCIM_OK;
}

// ===========================================================================
// pmCIMb step 2 with splitting, over all groups; step 3 afterwards
// ===========================================================================
struct EigOut {
  std::vector<double2> lam;
  std::vector<int> root, prob;
  std::vector<int64_t> vec_off;  // double2 offset of the eigenvector in ws.gdst
  size_t vec_used = 0;           // double2 entries used in ws.gdst
};

int run_beyn_levels(Call& c, const std::vector<HostRegion>& top, bool gate_top, EigOut* out,
                    std::vector<int>* root_status, std::vector<double>* top_ind, size_t n_roots = 0) {
  if (c.opt->indicator_N > 0)
    for (const HostRegion& h : top)
      if (h.N % c.opt->indicator_N)
        return fail(PMCIM_EINVAL, "N = %d is not a multiple of indicator_N = %d", h.N, c.opt->indicator_N);
  Workspace& ws = *c.ws;
  cudaStream_t s = c.s;
  std::vector<HostRegion> level = top;
  if (n_roots < top.size()) n_roots = top.size();
  root_status->assign(n_roots, 0);
  if (top_ind) top_ind->assign(n_roots, 0.0);
  const int Ni = c.opt->indicator_N;
  while (!level.empty()) {
    std::vector<HostRegion> next;
    std::vector<VecItem> vi;
    size_t vec_before = out->vec_used;
    int max_vn = 0;
    // eigenvectors of the last Beyn pass, from its scratch to the call's output
    // buffer (before the next pass overwrites the scratch)
    auto flush_vecs = [&]() -> int {
      if (vi.empty()) return PMCIM_OK;
      CU(ws.gdst.grow_keep(out->vec_used * sizeof(double2), vec_before * sizeof(double2), s));
      CU(ws.gitems.ensure(vi.size() * sizeof(VecItem)));
      CU(cudaMemcpyAsync(ws.gitems.p, vi.data(), vi.size() * sizeof(VecItem), cudaMemcpyHostToDevice, s));
      for (size_t q0 = 0; q0 < vi.size(); q0 += 65535) {
        const int cnt = (int)std::min<size_t>(65535, vi.size() - q0);
        prof_begin(PMCIM_K_GATHER, s);
        CU(launch_gather_vecs(ws.bvecs.as<double2>(), ws.gdst.as<double2>(), ws.gitems.as<VecItem>() + q0, cnt,
                              max_vn, s));
        prof_end(PMCIM_K_GATHER, s);
      }
      CU(cudaStreamSynchronize(s));
      vi.clear();
      vec_before = out->vec_used;
      max_vn = 0;
      return PMCIM_OK;
    };
    // node flags of the solves that ran
    auto node_flags = [&](const HostRegion& h, const RegionDev& d, const LevelOut& lo) {
      int& rs = (*root_status)[h.root];
      for (int j = 0; j < h.N; ++j) {
        const int v = lo.node_info[d.node_off + j];
        if (v & 0x00ffffff) {
          rs |= PMCIM_RS_SINGULAR_NODE;
          c.st.singular_nodes += 1;
        }
        if (v & (1 << 30)) rs |= PMCIM_RS_IR_FALLBACK;
      }
    };
    // Beyn's results of a disk: split it, or keep its filtered eigenvalues
    auto beyn_results = [&](const HostRegion& h, const RegionDev& d, const LevelOut& lo, int g) {
      int& rs = (*root_status)[h.root];
      if (lo.p[g] < 0) return;  // gated out
      c.st.candidates += 1;
      const int bits = lo.status[g];
      if ((bits & PMCIM_RS_SATURATED) && h.depth < c.opt->max_split_depth) {
        rs |= PMCIM_RS_SATURATED | PMCIM_RS_SPLIT;
        c.st.splits += 1;
        const double rc = h.r / 2.0, dd = rc / std::sqrt(2.0);
        const int sx[4] = {1, -1, 1, -1}, sy[4] = {1, 1, -1, -1};
        for (int q = 0; q < 4; ++q)
          next.push_back(HostRegion{h.cre + sx[q] * dd, h.cim + sy[q] * dd, rc, h.N, h.depth + 1, h.root, h.prob});
        return;
      }
      rs |= bits;
      const int n = c.pd[h.prob].n;
      for (int k = 0; k < lo.p[g]; ++k) {
        if (!lo.kept[(size_t)g * PMCIM_MAX_L + k]) continue;
        out->lam.push_back(lo.lam[(size_t)g * PMCIM_MAX_L + k]);
        out->root.push_back(h.root);
        out->prob.push_back(h.prob);
        out->vec_off.push_back((int64_t)out->vec_used);
        vi.push_back(VecItem{d.v_off + (int64_t)k * n, (int64_t)out->vec_used, n, 0});
        out->vec_used += (size_t)n;
        max_vn = std::max(max_vn, n);
      }
    };
    if (Ni <= 0) {
      // one N per disk: the level's solves feed the indicator and Beyn
      LevelOut lo;
      CHK(run_level(c, level, gate_top, true, &lo));
      for (int g = 0; g < (int)level.size(); ++g) {
        const HostRegion& h = level[g];
        node_flags(h, lo.rd[g], lo);
        if (h.depth == 0 && top_ind) (*top_ind)[h.root] = lo.ind[g];
        if (lo.cand[g]) (*root_status)[h.root] |= PMCIM_RS_CANDIDATE;
        beyn_results(h, lo.rd[g], lo, g);
      }
      CHK(flush_vecs());
    } else {
      // two passes (Appendix pmCIMb driver): the indicator on an Ni-node rule,
      // whose nodes are every (N / Ni)-th node of the disk's rule, then Beyn on the
      // candidates with the full rule, reusing the indicator pass's solutions.
      // Disks that the indicator does not gate (depth 0 without gate_top) go
      // straight to Beyn. Chunks bound the kept solutions.
      for (size_t q0 = 0; q0 < level.size();) {
        size_t q1 = q0, bytes = 0;
        while (q1 < level.size() && q1 - q0 < 65535) {
          const ProblemDev& P = c.pd[level[q1].prob];
          const size_t b = (size_t)Ni * P.n * P.l * sizeof(double2);
          if (q1 > q0 && bytes + b > kKeepBytes) break;
          bytes += b;
          ++q1;
        }
        std::vector<HostRegion> A;
        std::vector<size_t> a_of;
        for (size_t q = q0; q < q1; ++q)
          if (level[q].depth > 0 || gate_top) {
            A.push_back(level[q]);
            A.back().N = Ni;
            a_of.push_back(q);
          }
        LevelOut la;
        if (!A.empty()) CHK(run_level(c, A, false, false, &la, nullptr, false, nullptr, true));
        std::vector<HostRegion> B;
        LevelReuse ru;
        ru.X = ws.Xkeep.as<double2>();
        size_t ai = 0;
        for (size_t q = q0; q < q1; ++q) {
          const HostRegion& h = level[q];
          if (ai < a_of.size() && a_of[ai] == q) {
            const int g = (int)ai++;
            node_flags(A[g], la.rd[g], la);
            if (h.depth == 0 && top_ind) (*top_ind)[h.root] = la.ind[g];
            if (!la.cand[g]) continue;
            (*root_status)[h.root] |= PMCIM_RS_CANDIDATE;
            B.push_back(h);
            ru.src.push_back(la.rd[g].x_off);
            ru.stride.push_back(h.N / Ni);
          } else {
            B.push_back(h);
            ru.src.push_back(-1);
            ru.stride.push_back(1);
          }
        }
        if (!B.empty()) {
          LevelOut lb;
          CHK(run_level(c, B, false, true, &lb, nullptr, false, &ru, false, true));
          for (int g = 0; g < (int)B.size(); ++g) {
            const HostRegion& h = B[g];
            node_flags(h, lb.rd[g], lb);
            if (ru.src[g] < 0) {
              if (h.depth == 0 && top_ind) (*top_ind)[h.root] = lb.ind[g];
              if (lb.cand[g]) (*root_status)[h.root] |= PMCIM_RS_CANDIDATE;
            }
            beyn_results(h, lb.rd[g], lb, g);
          }
          CHK(flush_vecs());
        }
        q0 = q1;
      }
    }
    level.swap(next);
  }
  return PMCIM_OK;
}

// sigma_min (full) for the given values; slots sized for the largest n among them.
int run_verify(Call& c, const std::vector<double2>& lam, const std::vector<int>& prob, std::vector<double>* sig,
               std::vector<uint8_t>* acc, std::vector<double2>* vecs = nullptr, int* vec_stride = nullptr) {
  Workspace& ws = *c.ws;
  cudaStream_t s = c.s;
  const int m = (int)lam.size();
  sig->assign(m, 0.0);
  acc->assign(m, 0);
  if (m == 0) return PMCIM_OK;
  int max_n = 1;
  for (int i = 0; i < m; ++i) max_n = std::max(max_n, c.pd[prob[i]].n);
  const size_t slot = (size_t)max_n * max_n * sizeof(double2);
  const int slots = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>(2 * num_sms(), kSlotBytes / slot), m));
  CU(ws.vlam.ensure(m * sizeof(double2)));
  CU(ws.vprob.ensure(m * sizeof(int32_t)));
  CU(ws.vsig.ensure(m * sizeof(double)));
  CU(ws.vacc.ensure(m));
  CU(ws.vwork.ensure((size_t)slots * slot));
  CU(ws.vvec.ensure((size_t)slots * 3 * max_n * sizeof(double2)));
  CU(ws.vpiv.ensure((size_t)slots * max_n * sizeof(int32_t)));
  std::vector<int32_t> pr(prob.begin(), prob.end());
  CU(cudaMemcpyAsync(ws.vlam.p, lam.data(), m * sizeof(double2), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ws.vprob.p, pr.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  ValueArgs va;
  std::memset(&va, 0, sizeof(va));
  va.bie = any_bie(c.groups) ? 1 : 0;
  va.probs = ws.probs.as<ProblemDev>();
  va.prob_of = ws.vprob.as<int32_t>();
  va.lam = ws.vlam.as<double2>();
  va.m = m;
  va.tol_verify = c.opt->tol_verify;
  va.sigma = ws.vsig.as<double>();
  va.accept = ws.vacc.as<uint8_t>();
  va.work = ws.vwork.as<double2>();
  va.vec = ws.vvec.as<double2>();
  va.piv = ws.vpiv.as<int32_t>();
  va.slots = slots;
  va.max_n = max_n;
  if (vecs) {
    CU(ws.vout.ensure((size_t)m * max_n * sizeof(double2)));
    va.vec_out = ws.vout.as<double2>();
  }
  prof_begin(PMCIM_K_VERIFY, s);
  CU(launch_verify_fp64(va, s));
  prof_end(PMCIM_K_VERIFY, s);
  CU(cudaMemcpyAsync(sig->data(), ws.vsig.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(acc->data(), ws.vacc.p, m, cudaMemcpyDeviceToHost, s));
  if (vecs) {
    vecs->resize((size_t)m * max_n);
    *vec_stride = max_n;
    CU(cudaMemcpyAsync(vecs->data(), ws.vout.p, (size_t)m * max_n * sizeof(double2), cudaMemcpyDeviceToHost, s));
  }
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

// Certificate sigma_min(T(lambda)) <= ||T(lambda) v|| with the gathered unit eigenvectors.
// For problems with 1 to gram_max_dense() dense terms the products A_d v_i of all the
// call's values of a problem are formed at once (each A_d read once) and the norms
// ||T(lambda)||_F come from the coefficients' Gram data; otherwise one CTA per value
// forms T(lambda) element by element.
int run_certify(Call& c, const EigOut& e, std::vector<double>* cert, std::vector<uint8_t>* ok) {
  Workspace& ws = *c.ws;
  cudaStream_t s = c.s;
  const int m = (int)e.lam.size();
  cert->assign(m, 0.0);
  ok->assign(m, 0);
  if (m == 0) return PMCIM_OK;
  CU(ws.vlam.ensure(m * sizeof(double2)));
  CU(ws.vprob.ensure(m * sizeof(int32_t)));
  CU(ws.voff.ensure(m * sizeof(int64_t)));
  CU(ws.vsig.ensure(m * sizeof(double)));
  CU(ws.vacc.ensure(m));
  std::vector<int32_t> pr(e.prob.begin(), e.prob.end());
  CU(cudaMemcpyAsync(ws.vlam.p, e.lam.data(), m * sizeof(double2), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ws.vprob.p, pr.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ws.voff.p, e.vec_off.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  ValueArgs va;
  std::memset(&va, 0, sizeof(va));
  va.bie = any_bie(c.groups) ? 1 : 0;
  va.probs = ws.probs.as<ProblemDev>();
  va.prob_of = ws.vprob.as<int32_t>();
  va.lam = ws.vlam.as<double2>();
  va.vec_off = ws.voff.as<int64_t>();
  va.vecs = ws.gdst.as<double2>();
  va.m = m;
  va.tol_verify = c.opt->tol_verify;
  va.sigma = ws.vsig.as<double>();
  va.accept = ws.vacc.as<uint8_t>();
  bool products = true;
  for (const Group& g : c.groups)
    products = products && g.h->n_dense >= 1 && g.h->n_dense <= gram_max_dense() && !g.h->dG;
  prof_begin(PMCIM_K_VERIFY, s);
  if (products) {
    const size_t G = c.groups.size(), ge = gram_entries();
    // each problem's values in call order: W columns, vector offsets
    std::vector<std::vector<int>> of(G);
    for (int i = 0; i < m; ++i) of[e.prob[i]].push_back(i);
    std::vector<int64_t> w_col(m), order_off;
    std::vector<int32_t> w_m(m);
    std::vector<size_t> w_base(G), v_base(G);
    size_t wt = 0;
    for (size_t q = 0; q < G; ++q) {
      w_base[q] = wt;
      v_base[q] = order_off.size();
      const int mq = (int)of[q].size(), nq = c.pd[q].n;
      for (int k = 0; k < mq; ++k) {
        const int i = of[q][k];
        w_col[i] = (int64_t)(wt + (size_t)k * nq);
        w_m[i] = mq;
        order_off.push_back(e.vec_off[i]);
      }
      wt += (size_t)c.groups[q].h->n_dense * nq * mq;
    }
    CU(ws.cW.ensure(std::max<size_t>(1, wt) * sizeof(double2)));
    CU(ws.cidx.ensure((size_t)m * (2 * sizeof(int64_t) + sizeof(int32_t))));
    CU(ws.cgram.ensure(G * ge * sizeof(double2)));
    int64_t* d_order = ws.cidx.as<int64_t>();
    int64_t* d_wcol = d_order + m;
    int32_t* d_wm = reinterpret_cast<int32_t*>(d_wcol + m);
    CU(cudaMemcpyAsync(d_order, order_off.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d_wcol, w_col.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d_wm, w_m.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    for (size_t q = 0; q < G; ++q) {
      pmcim_problem h = c.groups[q].h;
      const ProblemDev* pq = ws.probs.as<ProblemDev>() + q;
      if (!h->gram_ok) {
        CU(h->gram.ensure(ge * sizeof(double2)));
        CU(ws.gpart.ensure(gram_partial_count() * ge * sizeof(double2)));
        CU(launch_gram(pq, ws.gpart.as<double2>(), h->gram.as<double2>(), s));
        h->gram_ok = true;
      }
      CU(cudaMemcpyAsync(ws.cgram.as<double2>() + q * ge, h->gram.p, ge * sizeof(double2),
                         cudaMemcpyDeviceToDevice, s));
      if (!of[q].empty())
        CU(launch_apply_dense(pq, c.pd[q].n, h->n_dense, ws.gdst.as<double2>(), d_order + v_base[q],
                              (int)of[q].size(), ws.cW.as<double2>() + w_base[q], s));
    }
    CU(launch_certify_products(va, ws.cW.as<double2>(), d_wcol, d_wm, ws.cgram.as<double2>(), s));
  } else {
    CU(launch_certify(va, s));
  }
  prof_end(PMCIM_K_VERIFY, s);
  CU(cudaMemcpyAsync(cert->data(), ws.vsig.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(ok->data(), ws.vacc.p, m, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

// One bordered inverse-iteration step with T(lambda)^H for the values whose
// eigenvector certificate did not accept them, in the manner of Dongarra, Moler
// and Wilkinson (SIAM J. Numer. Anal. 20, 1983): a low-precision factorisation,
// residuals in high precision. With the start vector c (Beyn's eigenvector) and
// s = argmax |c_i|, the node kernel solves M u = b, b = -T^H e_s, where M is
// T(lambda)^H with column s replaced by alpha c (k_border_rhs): the FP32 LU of M,
// residuals b - M X in FP64 (T^H assembled in FP64 once per value), FP32
// correction solves. T(lambda) is nearly singular at an eigenvalue, where a plain
// refinement cannot converge; M is not, so this one does. y = e_s + (u - u_s e_s)
// then satisfies T^H y = -u_s alpha c: y is the exact step T(lambda)^-H c, scaled
// to y_s = 1, and its residual is that of the exact step, not the FP32
// factorisation's backward error. The certificate is ||T^H y|| / ||y||, evaluated
// in FP64 from the coefficients; sigma_min(T^H) = sigma_min(T) <= ||T^H y|| / ||y||
// for every y != 0, however y was obtained, so a value whose certificate is at or
// below the acceptance threshold is accepted exactly as the sigma_min rule would
// accept it. Why T^H: with the singular value decomposition T = sum_k sigma_k u_k
// v_k^H, the step gives ||c|| / ||T^-H c||, about sigma_min / |v_min^H c|; Beyn's
// c approximates the right null vector v_min, so the certificate comes within a
// few digits of sigma_min. A step with T itself gives about sigma_min / |u_min^H c|
// and misses by the angle between the left and right null vectors. Each value is a
// pseudo-disk with one node z_0 = lambda (centre lambda, radius 0) and its own
// one-column problem entry; the values run in parallel, one per CTA. Problems with
// n <= 32 take the warp-per-node FP64 kernel, which solves T^H x = c directly (an
// FP64 solve already gives the exact step's residual).
int run_bordered_step(Call& c, const std::vector<double2>& lam_in, const std::vector<int>& prob_in,
                      const double2* start, const std::vector<int64_t>& start_off, std::vector<double>* cert,
                      std::vector<uint8_t>* ok) {
  Workspace& ws = *c.ws;
  cudaStream_t s = c.s;
  const int m = (int)lam_in.size();
  cert->assign(m, 0.0);
  ok->assign(m, 0);
  if (m == 0) return PMCIM_OK;
  std::vector<ProblemDev> pdv(m);
  std::vector<RegionDev> rdv(m);
  std::vector<NodeItem> it32, itS;
  std::vector<int32_t> prob_of(m);
  std::vector<int64_t> x_off(m), b_off(m, -1);
  size_t x_tot = 0, b_tot = 0;
  int max_n = 1, t64_n = 0;
  // the bordered right-hand sides and replacement columns: 2 n per value
  for (int i = 0; i < m; ++i) {
    const int n = c.pd[prob_in[i]].n;
    if (!small_kernel_fits(n, 1)) {
      b_off[i] = (int64_t)b_tot;
      b_tot += 2 * (size_t)n;
    }
  }
  CU(ws.ibord.ensure(std::max<size_t>(1, b_tot) * sizeof(double2)));
  const double2* bord = ws.ibord.as<double2>();
  for (int i = 0; i < m; ++i) {
    const int q = prob_in[i];
    pdv[i] = c.pd[q];
    pdv[i].l = 1;
    const int n = pdv[i].n;
    RegionDev& d = rdv[i];
    std::memset(&d, 0, sizeof(d));
    d.cre = lam_in[i].x;
    d.cim = lam_in[i].y;
    d.r = 0.0;
    d.N = 1;
    d.prob = i;
    d.node_off = i;
    d.lu_tc = 1;
    d.herm = 1;
    d.x_off = (int64_t)x_tot;
    x_off[i] = (int64_t)x_tot;
    x_tot += (size_t)n;
    prob_of[i] = q;
    max_n = std::max(max_n, n);
    if (b_off[i] < 0) {
      pdv[i].V = start + start_off[i];  // T(lambda)^H x = c in FP64
      itS.push_back(NodeItem{i, 0});
    } else {
      pdv[i].V = bord + b_off[i];       // b; the column alpha c follows it
      d.v_off = b_off[i] + n;           // d.border is set on the device
      it32.push_back(NodeItem{i, 0});
      t64_n = std::max(t64_n, n);  // T^H in FP64 for the residuals
    }
  }
  std::stable_sort(it32.begin(), it32.end(), [&](const NodeItem& a, const NodeItem& b) {
    return pdv[a.region].n != pdv[b.region].n ? pdv[a.region].n > pdv[b.region].n : a.region < b.region;
  });
  std::vector<NodeItem> items(it32);
  items.insert(items.end(), itS.begin(), itS.end());
  CU(ws.iprobs.ensure(m * sizeof(ProblemDev)));
  CU(ws.iregions.ensure(m * sizeof(RegionDev)));
  CU(ws.iitems.ensure(items.size() * sizeof(NodeItem)));
  CU(ws.iX.ensure(x_tot * sizeof(double2)));
  CU(ws.iinfo.ensure(m * sizeof(int32_t)));
  CU(ws.icounters.ensure(4 * sizeof(int32_t)));
  CU(ws.ioffs.ensure((size_t)m * 2 * sizeof(int64_t)));
  CU(ws.vlam.ensure(m * sizeof(double2)));
  CU(ws.vprob.ensure(m * sizeof(int32_t)));
  CU(ws.voff.ensure(m * sizeof(int64_t)));
  CU(ws.vsig.ensure(m * sizeof(double)));
  CU(ws.vacc.ensure(m));
  int64_t* d_start_off = ws.ioffs.as<int64_t>();
  int64_t* d_b_off = d_start_off + m;
  CU(cudaMemcpyAsync(ws.iprobs.p, pdv.data(), m * sizeof(ProblemDev), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ws.iregions.p, rdv.data(), m * sizeof(RegionDev), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ws.iitems.p, items.data(), items.size() * sizeof(NodeItem), cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(ws.icounters.p, 0, 4 * sizeof(int32_t), s));
  CU(cudaMemcpyAsync(ws.vlam.p, lam_in.data(), m * sizeof(double2), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ws.vprob.p, prob_of.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d_start_off, start_off.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d_b_off, b_off.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  ValueArgs va;
  std::memset(&va, 0, sizeof(va));
  va.bie = any_bie(c.groups) ? 1 : 0;
  va.probs = ws.probs.as<ProblemDev>();
  va.prob_of = ws.vprob.as<int32_t>();
  va.lam = ws.vlam.as<double2>();
  va.m = m;
  va.tol_verify = c.opt->tol_verify;
  va.sigma = ws.vsig.as<double>();
  va.accept = ws.vacc.as<uint8_t>();
  va.herm = 1;
  if (!it32.empty()) {
    va.vec_off = d_start_off;
    va.vecs = start;
    prof_begin(PMCIM_K_VERIFY, s);
    CU(launch_border_rhs(va, d_b_off, ws.ibord.as<double2>(), ws.iregions.as<RegionDev>(), s));
    prof_end(PMCIM_K_VERIFY, s);
  }
  NodeArgs na;
  std::memset(&na, 0, sizeof(na));
  na.bie = any_bie(c.groups) ? 1 : 0;
  na.probs = ws.iprobs.as<ProblemDev>();
  na.regions = ws.iregions.as<RegionDev>();
  na.X = ws.iX.as<double2>();
  na.node_info = ws.iinfo.as<int32_t>();
  na.max_n = max_n;
  na.max_sweeps = std::max(1, c.opt->max_ir_sweeps);
  na.tol_ir = kIrTol;
  na.err = ws.icounters.as<int32_t>() + 3;
  na.tc_wait_cycles = wait_limit_tc();
  na.handoff_wait_cycles = wait_limit_handoff();
  na.border = bord;
  const int sms = num_sms();
  if (!it32.empty()) {
    const size_t slot32 = mixed_slot_bytes(max_n, 1);
    const size_t per = (size_t)mixed_slots_per_cta();
    const size_t t64_stride = (size_t)t64_n * t64_n;
    const size_t cta_bytes = per * (slot32 + t64_stride * sizeof(double2));
    const size_t budget = slot_budget(ws.work32.cap + ws.t64.cap);
    // one value per CTA (its other slot idle): the values are few, and a CTA works
    // through its slots one node after another
    const size_t ctas = std::max<size_t>(1, std::min<size_t>(std::min<size_t>(sms, budget / cta_bytes),
                                                             it32.size()));
    const int slots32 = (int)(ctas * per);
    CU(ws.work32.ensure((size_t)slots32 * slot32));
    CU(ws.piv32.ensure((size_t)slots32 * max_n * sizeof(int32_t)));
    CU(ws.t64.ensure((size_t)slots32 * t64_stride * sizeof(double2)));
    CU(prepare_factor_mixed());
    na.oz = 0;
    na.ysl = nullptr;
    na.ysl_stride = 0;
    na.items = ws.iitems.as<NodeItem>();
    na.n_items = (int)it32.size();
    na.counter = ws.icounters.as<int>() + 1;
    na.work = ws.work32.as<char>();
    na.slot_bytes = slot32;
    na.piv = ws.piv32.as<int32_t>();
    na.slots = slots32;
    na.t64 = ws.t64.as<double2>();
    na.t64_stride = t64_stride;
    na.phase = nullptr;
    prof_begin(PMCIM_K_VERIFY, s);  // verification work, timed apart from the disks' nodes
    CU(launch_factor_solve_mixed(na, s));
    prof_end(PMCIM_K_VERIFY, s);
  }
  if (!itS.empty()) {
    CU(prepare_factor_small());
    na.items = ws.iitems.as<NodeItem>() + it32.size();
    na.n_items = (int)itS.size();
    na.counter = ws.icounters.as<int>() + 2;
    prof_begin(PMCIM_K_VERIFY, s);
    CU(launch_factor_solve_small(na, s));
    prof_end(PMCIM_K_VERIFY, s);
  }
  // the certificate of y, against the call's own problem table
  CU(cudaMemcpyAsync(ws.voff.p, x_off.data(), m * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  va.vec_off = ws.voff.as<int64_t>();
  va.vecs = ws.iX.as<double2>();
  prof_begin(PMCIM_K_VERIFY, s);
  CU(launch_certify(va, s));
  prof_end(PMCIM_K_VERIFY, s);
  int32_t handoff_err = 0;
  CU(cudaMemcpyAsync(cert->data(), ws.vsig.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(ok->data(), ws.vacc.p, m, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(&handoff_err, ws.icounters.as<int32_t>() + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (handoff_err)
    return fail(PMCIM_ETIMEOUT, "precision-form node kernel: a wait between its thread groups ran out");
  // a value whose certificate is not finite (e.g. an exactly singular T(lambda)) is left
  // to the full sigma_min computation
  for (int i = 0; i < m; ++i)
    if (!std::isfinite((*cert)[i])) (*ok)[i] = 0;
  return PMCIM_OK;
}

// Steps 1-3 for all groups of a call. Outputs in call order (not sorted).
struct Verified {
  std::vector<double> sig;
  std::vector<uint8_t> acc;
};

// Learned screen: coarse indicators of every disk (one probe column, screen_N
// nodes), the MLP's probabilities, and the disks that may skip the full path.
int run_screen(Call& c, const std::vector<HostRegion>& top, std::vector<uint8_t>* skip) {
  Workspace& ws = *c.ws;
  cudaStream_t s = c.s;
  const int R = (int)top.size();
  skip->assign(R, 0);
  if (R == 0) return PMCIM_OK;
  const int NS = c.opt->screen_N > 0 ? c.opt->screen_N : 16;
  if (NS % 16) return fail(PMCIM_EINVAL, "screen_N = %d is not a multiple of 16", NS);
  // coarse copies of the groups: same coefficients and probe block, one column
  const size_t G = c.groups.size();
  for (size_t gi = 0; gi < G; ++gi)
    c.groups.push_back(Group{c.groups[gi].h, 1, c.groups[gi].form, c.groups[gi].tile});
  CHK(upload_problems(c));
  std::vector<HostRegion> coarse = top;
  for (HostRegion& h : coarse) {
    h.N = NS;
    h.prob += (int)G;
  }
  LevelOut lo;
  CHK(run_level(c, coarse, false, false, &lo, nullptr, true));
  c.st.screen_solves += (int)(R * NS);
  c.st.solves -= (int64_t)R * NS;  // counted as screen work, not as pmCIMb solves
  c.st.regions -= R;
  CU(ws.sparams.ensure(PMCIM_SCREEN_PARAMS * sizeof(float)));
  CU(ws.sscratch.ensure(2 * PMCIM_SCREEN_PARAMS + 256));
  CU(ws.sprob.ensure(R * sizeof(float)));
  CU(cudaMemcpyAsync(ws.sparams.p, c.opt->screen_params, PMCIM_SCREEN_PARAMS * sizeof(float), cudaMemcpyDefault, s));
  prof_begin(PMCIM_K_SCREEN, s);
  CU(screen_forward(R, ws.feats.as<float>(), ws.sparams.as<float>(), ws.sprob.as<float>(), ws.sscratch.p, s));
  prof_end(PMCIM_K_SCREEN, s);
  std::vector<float> prob(R);
  std::vector<double> ind3((size_t)R * 3);
  CU(cudaMemcpyAsync(prob.data(), ws.sprob.p, R * sizeof(float), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(ind3.data(), ws.ind3.p, (size_t)R * 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  // skip only a confident negative: the network below its threshold AND both
  // coarse indicators (Eq. 3.1 with 8 and 16 nodes) at or below tol_ind, so a
  // disk the paper's own coarse screen would flag is never dropped
  for (int g = 0; g < R; ++g)
    (*skip)[g] = (prob[g] < c.opt->screen_threshold && !(ind3[3 * (size_t)g] > c.opt->tol_ind) &&
                  !(ind3[3 * (size_t)g + 1] > c.opt->tol_ind))
                     ? 1
                     : 0;
  c.groups.resize(G);
  CHK(upload_problems(c));
  return PMCIM_OK;
}

int run_pmcimb(Call& c, const std::vector<HostRegion>& top_in, EigOut* e, Verified* v, std::vector<int>* rstat,
               std::vector<double>* tind) {
  CHK(tune_forms(c));
  std::vector<HostRegion> top = top_in;
  std::vector<uint8_t> skip;
  if (c.opt->screen_params) {
    CHK(run_screen(c, top_in, &skip));
    top.clear();
    for (size_t g = 0; g < top_in.size(); ++g)
      if (!skip[g]) top.push_back(top_in[g]);
      else c.st.screened_out += 1;
  }
  CHK(run_beyn_levels(c, top, true, e, rstat, tind, top_in.size()));
  if (!skip.empty())
    for (size_t g = 0; g < top_in.size(); ++g)
      if (skip[g]) {
        (*rstat)[top_in[g].root] |= PMCIM_RS_SCREENED;
        if (tind) (*tind)[top_in[g].root] = -1.0;
      }
  CHK(run_certify(c, *e, &v->sig, &v->acc));
  std::vector<double2> rest;
  std::vector<int> rest_prob, idx;
  for (size_t i = 0; i < e->lam.size(); ++i) {
    if (v->acc[i]) {
      c.st.certified += 1;
    } else {
      rest.push_back(e->lam[i]);
      rest_prob.push_back(e->prob[i]);
      idx.push_back((int)i);
    }
  }
  // a second certificate from the bordered inverse step started at Beyn's vector (it runs
  // the precision form's node kernel, so values of boundary-integral problems skip it and
  // go to the full sigma_min below)
  {
    std::vector<double2> skip_lam;
    std::vector<int> skip_prob, skip_idx;
    {
      std::vector<double2> keep_lam;
      std::vector<int> keep_prob, keep_idx;
      for (size_t k = 0; k < idx.size(); ++k) {
        const bool bie = c.groups[rest_prob[k]].h->dG != nullptr;
        (bie ? skip_lam : keep_lam).push_back(rest[k]);
        (bie ? skip_prob : keep_prob).push_back(rest_prob[k]);
        (bie ? skip_idx : keep_idx).push_back(idx[k]);
      }
      rest.swap(keep_lam);
      rest_prob.swap(keep_prob);
      idx.swap(keep_idx);
    }
    std::vector<int64_t> start_off;
    for (int k : idx) start_off.push_back(e->vec_off[k]);
    std::vector<double> cert2;
    std::vector<uint8_t> ok2;
    CHK(run_bordered_step(c, rest, rest_prob, c.ws->gdst.as<double2>(), start_off, &cert2, &ok2));
    std::vector<double2> rest2;
    std::vector<int> rest2_prob, idx2;
    for (size_t k = 0; k < idx.size(); ++k) {
      if (ok2[k]) {
        v->sig[idx[k]] = cert2[k];
        v->acc[idx[k]] = 1;
        c.st.certified += 1;
      } else {
        rest2.push_back(rest[k]);
        rest2_prob.push_back(rest_prob[k]);
        idx2.push_back(idx[k]);
      }
    }
    rest.swap(rest2);
    rest_prob.swap(rest2_prob);
    idx.swap(idx2);
    rest.insert(rest.end(), skip_lam.begin(), skip_lam.end());
    rest_prob.insert(rest_prob.end(), skip_prob.begin(), skip_prob.end());
    idx.insert(idx.end(), skip_idx.begin(), skip_idx.end());
  }
  std::vector<double> sig2;
  std::vector<uint8_t> acc2;
  CHK(run_verify(c, rest, rest_prob, &sig2, &acc2));
  for (size_t k = 0; k < idx.size(); ++k) {
    v->sig[idx[k]] = sig2[k];
    v->acc[idx[k]] = acc2[k];
  }
  for (size_t i = 0; i < e->lam.size(); ++i)
    if (!v->acc[i]) c.st.unverified += 1;
  return PMCIM_OK;
}

std::vector<HostRegion> to_host_regions(int R, const pmcim_region* reg, int prob, int root0 = 0) {
  std::vector<HostRegion> v(R);
  for (int g = 0; g < R; ++g) v[g] = HostRegion{reg[g].c_re, reg[g].c_im, reg[g].r, reg[g].N, 0, root0 + g, prob};
  return v;
}

int check_device() {
  int cnt = 0;
  cudaError_t e = cudaGetDeviceCount(&cnt);
  if (e != cudaSuccess || cnt == 0) return fail(PMCIM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  return PMCIM_OK;
}

int single_call(Call& c, pmcim_problem p, const pmcim_options* opt, int l, const double* V) {
  c.opt = opt;
  c.ws = &p->ws;
  CHK(call_stream(p->ws, opt, &c.s));
  const int form = opt->precision == PMCIM_PREC_AUTO ? PMCIM_PREC_FP32_IR : opt->precision;
  c.groups = {Group{p, l, form, opt->fp64_tile ? opt->fp64_tile : 64}};
  CHK(upload_V(p, l, V, c.s));
  CHK(upload_problems(c));
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
  opt->max_ir_sweeps = 6;
  opt->max_split_depth = 8;
  opt->cuda_stream = nullptr;
  opt->screen_params = nullptr;
  opt->screen_threshold = 0.0;
  opt->screen_N = 16;
  opt->tol_ir = kIrTol;
  opt->beyn_K = 1;
  opt->residual_fp64 = 0;
  opt->fp64_tile = 0;
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
  for (int q = 0; q < PMCIM_PHASE_COUNT; ++q) P.phase[q] = 0.0;
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
  for (int q = 0; q < PMCIM_PHASE_COUNT; ++q) out->mixed_phase_cycles[q] = P.phase[q];
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
  int nd = 0, n_bie = 0;
  for (int k = 0; k < K; ++k) {
    if (f[k].kind != PMCIM_F_MONOMIAL && f[k].kind != PMCIM_F_EXP_NEG && f[k].kind != PMCIM_F_HELMHOLTZ_DLP) {
      delete p;
      return fail(PMCIM_EINVAL, "term %d: unknown kind %d", k, f[k].kind);
    }
    if (f[k].kind == PMCIM_F_HELMHOLTZ_DLP) {
      if (!A[k] || ++n_bie > 1) {
        delete p;
        return fail(PMCIM_EINVAL, "term %d: a boundary-integral term needs its curve, and one such term at most", k);
      }
      TermDesc& t = p->term[k];
      t.kind = f[k].kind;
      t.degree = 0;
      t.tau = 0.0;
      t.id = make_double2(f[k].id_re, f[k].id_im);
      t.dense = 0;
      t.mat_index = -1;
      // the curve's samples (host or device) -> the device geometry of bie.cuh
      std::vector<double> smp((size_t)6 * n), G((size_t)6 * n + 1);
      cudaError_t e = cudaMemcpy(smp.data(), A[k], smp.size() * sizeof(double), cudaMemcpyDefault);
      if (e != cudaSuccess) {
        delete p;
        return fail(PMCIM_ECUDA, "curve copy: %s", cudaGetErrorString(e));
      }
      if (!bie::build_geometry(smp.data(), n, G.data())) {
        delete p;
        return fail(PMCIM_EINVAL, "term %d: the curve needs an even n >= 4 and finite, distinct samples with "
                                  "x' != 0", k);
      }
      p->bie_circ = G[(size_t)6 * n] != 0.0;
      e = cudaMalloc(&p->dG, G.size() * sizeof(double));
      if (e == cudaSuccess) e = cudaMemcpy(p->dG, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        if (p->dG) cudaFree(p->dG);
        delete p;
        return fail(PMCIM_ENOMEM, "curve upload: %s", cudaGetErrorString(e));
      }
      continue;
    }
    if (f[k].kind == PMCIM_F_MONOMIAL && (f[k].degree < 0 || f[k].degree > 16)) {
      delete p;
      return fail(PMCIM_EINVAL, "term %d: degree %d outside 0..16", k, f[k].degree);
    }
    TermDesc& t = p->term[k];
    t.kind = f[k].kind;
    t.degree = f[k].degree;
    t.tau = f[k].tau;
    t.id = make_double2(f[k].id_re, f[k].id_im);
    t.dense = A[k] ? 1 : 0;
    t.mat_index = A[k] ? nd++ : -1;
  }
  p->n_dense = nd;
  cudaGetDevice(&p->device);
  const size_t nn = (size_t)n * n;
  if (nd > 0) {
    cudaError_t e = cudaMalloc(&p->dA, (size_t)nd * nn * sizeof(double2));
    if (e != cudaSuccess) {
      if (p->dG) cudaFree(p->dG);
      delete p;
      return fail(PMCIM_ENOMEM, "coefficient upload: %s", cudaGetErrorString(e));
    }
    for (int k = 0; k < K; ++k) {
      if (!A[k]) continue;
      e = cudaMemcpy(p->dA + (size_t)p->term[k].mat_index * nn, A[k], nn * sizeof(double2), cudaMemcpyDefault);
      if (e != cudaSuccess) {
        cudaFree(p->dA);
        if (p->dG) cudaFree(p->dG);
        delete p;
        return fail(PMCIM_ECUDA, "coefficient upload: %s", cudaGetErrorString(e));
      }
    }
    e = cudaMalloc(&p->dA32, (size_t)nd * nn * sizeof(float2));
    if (e == cudaSuccess) e = round_coefficients_c64(p->dA, p->dA32, (size_t)nd * nn, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaFree(p->dA);
      if (p->dA32) cudaFree(p->dA32);
      if (p->dG) cudaFree(p->dG);
      delete p;
      return fail(PMCIM_ENOMEM, "coefficient copy: %s", cudaGetErrorString(e));
    }
  }
  *out = p;
  return PMCIM_OK;
}

int pmcim_problem_destroy(pmcim_problem p) {
  if (!p) return PMCIM_OK;
  cudaDeviceSynchronize();
  if (p->dA) cudaFree(p->dA);
  if (p->dA32) cudaFree(p->dA32);
  if (p->dG) cudaFree(p->dG);
  p->dig.release();
  p->dexp.release();
  p->V.release();
  p->ws.release();
  delete p;
  return PMCIM_OK;
}

int pmcim_moments(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
                  const double* V, double* C0, double* C1, double* pf_half, double* pf_abs) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l));
  Call c;
  CHK(single_call(c, p, opt, l, V));
  LevelOut lo;
  CHK(run_level(c, to_host_regions(R, reg, 0), false, false, &lo));
  const size_t nl = (size_t)p->n * l;
  if (C0) CHK(copy_out(C0, p->ws.C0.p, (size_t)R * nl * sizeof(double2)));
  if (C1) CHK(copy_out(C1, p->ws.C1.p, (size_t)R * nl * sizeof(double2)));
  if (pf_half) CHK(copy_out(pf_half, p->ws.pf_half.p, (size_t)R * p->n * sizeof(double2)));
  if (pf_abs) CHK(copy_out(pf_abs, p->ws.pf_abs.p, (size_t)R * p->n * sizeof(double)));
  return PMCIM_OK;
}

int pmcim_indicator(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
                    const double* V, double* ind, double* pf_norm, double* pf_scale, uint8_t* candidate) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l));
  if (R > 0 && (!ind || !candidate)) return fail(PMCIM_EINVAL, "ind or candidate is NULL");
  Call c;
  CHK(single_call(c, p, opt, l, V));
  LevelOut lo;
  CHK(run_level(c, to_host_regions(R, reg, 0), false, false, &lo));
  if (R > 0) {
    CHK(copy_out(ind, p->ws.ind.p, R * sizeof(double)));
    CHK(copy_out(candidate, p->ws.cand.p, R));
    if (pf_norm) CHK(copy_out(pf_norm, p->ws.pf_norm.p, R * sizeof(double)));
    if (pf_scale) CHK(copy_out(pf_scale, p->ws.pf_scale.p, R * sizeof(double)));
  }
  return PMCIM_OK;
}

int pmcim_beyn(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
               const double* V, int32_t cap, double* lambda, double* vecs, int32_t* region_of, int32_t* count,
               int32_t* region_status) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l));
  if (!count || cap < 0 || (cap > 0 && !lambda)) return fail(PMCIM_EINVAL, "bad output arguments");
  Call c;
  CHK(single_call(c, p, opt, l, V));
  EigOut out;
  std::vector<int> rstat;
  CHK(run_beyn_levels(c, to_host_regions(R, reg, 0), false, &out, &rstat, nullptr));
  const int cnt = (int)out.lam.size();
  CHK(copy_out(count, &cnt, sizeof(int32_t)));
  if (region_status) CHK(copy_out(region_status, rstat.data(), R * sizeof(int32_t)));
  if (cnt > cap) return fail(PMCIM_ECAPACITY, "%d eigenvalues exceed capacity %d", cnt, cap);
  CHK(copy_out(lambda, out.lam.data(), cnt * sizeof(double2)));
  if (region_of) CHK(copy_out(region_of, out.root.data(), cnt * sizeof(int32_t)));
  if (vecs && cnt > 0) CHK(copy_out(vecs, p->ws.gdst.p, (size_t)cnt * p->n * sizeof(double2)));
  return PMCIM_OK;
}

int pmcim_residual(pmcim_problem p, const pmcim_options* opt, int32_t m, const double* z, int32_t l,
                   const double* V, const double* X, double* R) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  if (m < 0 || l < 1 || l > PMCIM_MAX_L) return fail(PMCIM_EINVAL, "m = %d or l = %d out of range", m, l);
  if (m > 0 && (!z || !V || !X || !R)) return fail(PMCIM_EINVAL, "NULL buffer");
  if (p->dG) return fail(PMCIM_EINVAL, "the tensor-core residual needs coefficient matrices; this problem has a "
                                       "boundary-integral term");
  if (m == 0) return PMCIM_OK;
  Call c;
  c.opt = opt;
  c.ws = &p->ws;
  CHK(call_stream(p->ws, opt, &c.s));
  c.groups = {Group{p, l, PMCIM_PREC_FP32_IR}};
  CHK(upload_V(p, l, V, c.s));
  CHK(ensure_digits(p, c.s));
  CHK(upload_problems(c));
  Workspace& ws = p->ws;
  const size_t nl = (size_t)p->n * l;
  CU(ws.rz.ensure(m * sizeof(double2)));
  CU(ws.rX.ensure((size_t)m * nl * sizeof(double2)));
  CU(ws.rR.ensure((size_t)m * nl * sizeof(double2)));
  CU(ws.rstat.ensure(m * sizeof(int32_t)));
  const int ctas = std::min(num_sms(), (int)m);
  const size_t stride = y_digit_scratch_bytes(p->n, std::max(1, p->n_dense));
  CU(ws.rysl.ensure((size_t)ctas * stride));
  CU(cudaMemcpyAsync(ws.rz.p, z, m * sizeof(double2), cudaMemcpyDefault, c.s));
  CU(cudaMemcpyAsync(ws.rX.p, X, (size_t)m * nl * sizeof(double2), cudaMemcpyDefault, c.s));
  CU(launch_residual_points(ws.probs.as<ProblemDev>(), ws.rz.as<double2>(), m, ws.rX.as<double2>(),
                            ws.rR.as<double2>(), ws.rysl.as<unsigned char>(), stride, ctas, ws.rstat.as<int32_t>(),
                            wait_limit_tc(), c.s));
  std::vector<int32_t> st(m);
  CU(cudaMemcpyAsync(R, ws.rR.p, (size_t)m * nl * sizeof(double2), cudaMemcpyDefault, c.s));
  CU(cudaMemcpyAsync(st.data(), ws.rstat.p, m * sizeof(int32_t), cudaMemcpyDeviceToHost, c.s));
  CU(cudaStreamSynchronize(c.s));
  for (int i = 0; i < m; ++i)
    if (st[i]) return fail(PMCIM_ETIMEOUT, "residual at point %d: a tensor-core wait ran out", i);
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
  Call c;
  c.opt = opt;
  c.ws = &p->ws;
  CHK(call_stream(p->ws, opt, &c.s));
  c.groups = {Group{p, 1, PMCIM_PREC_FP64}};
  CHK(upload_problems(c));
  std::vector<double> sig;
  std::vector<uint8_t> acc;
  CHK(run_verify(c, lam, std::vector<int>(m, 0), &sig, &acc));
  CHK(copy_out(sigma_min, sig.data(), m * sizeof(double)));
  if (accept) CHK(copy_out(accept, acc.data(), m));
  return PMCIM_OK;
}

int pmcim_certify(pmcim_problem p, const pmcim_options* opt, int32_t m, const double* lambda, const double* vecs,
                  double* cert, uint8_t* accept) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  if (m < 0 || (m > 0 && (!lambda || !vecs || !cert))) return fail(PMCIM_EINVAL, "bad arguments");
  if (m == 0) return PMCIM_OK;
  const int n = p->n;
  std::vector<double2> lam(m);
  cudaError_t e = cudaMemcpy(lam.data(), lambda, m * sizeof(double2), cudaMemcpyDefault);
  if (e != cudaSuccess) return fail(PMCIM_ECUDA, "lambda copy: %s", cudaGetErrorString(e));
  Call c;
  c.opt = opt;
  c.ws = &p->ws;
  CHK(call_stream(p->ws, opt, &c.s));
  c.groups = {Group{p, 1, p->dG ? PMCIM_PREC_FP64
                                : opt->precision == PMCIM_PREC_AUTO ? PMCIM_PREC_FP32_IR : opt->precision}};
  CHK(upload_problems(c));
  Workspace& ws = p->ws;
  CU(ws.gdst.ensure((size_t)m * n * sizeof(double2)));
  CU(cudaMemcpyAsync(ws.gdst.p, vecs, (size_t)m * n * sizeof(double2), cudaMemcpyDefault, c.s));
  EigOut eo;
  eo.lam = lam;
  eo.prob.assign(m, 0);
  eo.root.assign(m, 0);
  for (int i = 0; i < m; ++i) eo.vec_off.push_back((int64_t)i * n);
  std::vector<double> sig;
  std::vector<uint8_t> acc;
  CHK(run_certify(c, eo, &sig, &acc));
  std::vector<double2> rest;
  std::vector<int64_t> off;
  std::vector<int> idx;
  for (int i = 0; i < m; ++i)
    if (!acc[i] || !std::isfinite(sig[i])) {
      acc[i] = 0;
      rest.push_back(lam[i]);
      off.push_back((int64_t)i * n);
      idx.push_back(i);
    }
  if (p->dG) {  // the bordered step runs the precision form's node kernel: coefficient problems only
    rest.clear();
    off.clear();
    idx.clear();
  }
  std::vector<double> sig2;
  std::vector<uint8_t> acc2;
  CHK(run_bordered_step(c, rest, std::vector<int>(rest.size(), 0), ws.gdst.as<double2>(), off, &sig2, &acc2));
  for (size_t k = 0; k < idx.size(); ++k) {
    const int i = idx[k];
    if (std::isfinite(sig2[k]) && !(sig2[k] >= sig[i])) sig[i] = sig2[k];
    acc[i] = acc2[k];
  }
  CHK(copy_out(cert, sig.data(), m * sizeof(double)));
  if (accept) CHK(copy_out(accept, acc.data(), m));
  return PMCIM_OK;
}

int pmcim_pmcima(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, const double* V,
                 double tol_eps, int32_t cap, double* lambda, double* vecs, double* sigma_min, int32_t* count,
                 pmcim_stats* stats) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, 1));
  if (!(tol_eps > 0.0) || !std::isfinite(tol_eps)) return fail(PMCIM_EINVAL, "tol_eps must be positive");
  if (!count || cap < 0 || (cap > 0 && !lambda)) return fail(PMCIM_EINVAL, "bad output arguments");
  Call c;
  CHK(single_call(c, p, opt, 1, V));
  CHK(tune_forms(c));
  // step 1: levels of indicators; candidates are quadrisected until the disk's level count
  std::vector<int> levels(R);
  for (int g = 0; g < R; ++g) levels[g] = std::max(1, (int)std::ceil(std::log2(reg[g].r / tol_eps)) + 2);
  std::vector<HostRegion> level = to_host_regions(R, reg, 0);
  std::vector<double2> centres;
  while (!level.empty()) {
    if (level.size() > kMaxPmcimaRegions)
      return fail(PMCIM_ECAPACITY, "pmCIMa level of %zu disks: the indicator marks too many disks",
                  level.size());
    LevelOut lo;
    CHK(run_level(c, level, false, false, &lo));
    std::vector<HostRegion> next;
    for (size_t g = 0; g < level.size(); ++g) {
      if (!lo.cand[g]) continue;
      const HostRegion& h = level[g];
      c.st.candidates += 1;
      if (h.depth + 1 < levels[h.root]) {
        const double rc = h.r / 2.0, dd = rc / std::sqrt(2.0);
        const int sx[4] = {1, -1, 1, -1}, sy[4] = {1, 1, -1, -1};
        for (int q = 0; q < 4; ++q)
          next.push_back(HostRegion{h.cre + sx[q] * dd, h.cim + sy[q] * dd, rc, h.N, h.depth + 1, h.root, h.prob});
      } else {
        centres.push_back(make_double2(h.cre, h.cim));
      }
    }
    level.swap(next);
  }
  // merge: in order, each free centre takes the free centres within tol_eps (itself once), mean
  std::vector<double2> lam;
  std::vector<uint8_t> used(centres.size(), 0);
  for (size_t i = 0; i < centres.size(); ++i) {
    if (used[i]) continue;
    double sr = 0.0, si = 0.0;
    int k = 0;
    for (size_t j = 0; j < centres.size(); ++j) {
      if (used[j] || std::hypot(centres[i].x - centres[j].x, centres[i].y - centres[j].y) >= tol_eps) continue;
      used[j] = 1;
      sr += centres[j].x;
      si += centres[j].y;
      ++k;
    }
    lam.push_back(make_double2(sr / k, si / k));
  }
  std::sort(lam.begin(), lam.end(), [](const double2& a, const double2& b) {
    return a.x != b.x ? a.x < b.x : a.y < b.y;
  });
  const int m = (int)lam.size();
  *count = m;
  if (stats) *stats = c.st;
  if (m > cap) return fail(PMCIM_ECAPACITY, "%d values, capacity %d", m, cap);
  // step 2: sigma_min of T(lambda) and its right singular vector
  std::vector<double> sig;
  std::vector<uint8_t> acc;
  std::vector<double2> vv;
  int stride = 0;
  CHK(run_verify(c, lam, std::vector<int>(m, 0), &sig, &acc, vecs ? &vv : nullptr, vecs ? &stride : nullptr));
  if (m > 0) {
    CHK(copy_out(lambda, lam.data(), m * sizeof(double2)));
    if (sigma_min) CHK(copy_out(sigma_min, sig.data(), m * sizeof(double)));
    if (vecs) {
      std::vector<double2> packed((size_t)m * p->n);
      for (int i = 0; i < m; ++i)
        std::memcpy(packed.data() + (size_t)i * p->n, vv.data() + (size_t)i * stride, p->n * sizeof(double2));
      CHK(copy_out(vecs, packed.data(), packed.size() * sizeof(double2)));
    }
  }
  if (stats) *stats = c.st;
  return PMCIM_OK;
}

int pmcim_solve(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg, int32_t l,
                const double* V, int32_t cap, double* lambda, double* vecs, double* sigma_min, int32_t* region_of,
                int32_t* count, double* ind, int32_t* region_status, pmcim_stats* stats) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l));
  if (!count || cap < 0 || (cap > 0 && !lambda)) return fail(PMCIM_EINVAL, "bad output arguments");
  Call c;
  CHK(single_call(c, p, opt, l, V));
  EigOut e;
  Verified v;
  std::vector<int> rstat;
  std::vector<double> tind;
  CHK(run_pmcimb(c, to_host_regions(R, reg, 0), &e, &v, &rstat, &tind));
  std::vector<int> order;
  for (size_t i = 0; i < e.lam.size(); ++i)
    if (v.acc[i]) order.push_back((int)i);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (e.lam[a].x != e.lam[b].x) return e.lam[a].x < e.lam[b].x;
    return e.lam[a].y < e.lam[b].y;
  });
  const int cnt = (int)order.size();
  CHK(copy_out(count, &cnt, sizeof(int32_t)));
  if (ind) CHK(copy_out(ind, tind.data(), R * sizeof(double)));
  if (region_status) CHK(copy_out(region_status, rstat.data(), R * sizeof(int32_t)));
  if (stats) CHK(copy_out(stats, &c.st, sizeof(c.st)));
  if (cnt > cap) return fail(PMCIM_ECAPACITY, "%d eigenvalues exceed capacity %d", cnt, cap);
  std::vector<double2> lam_s(cnt);
  std::vector<double> sig_s(cnt);
  std::vector<int32_t> root_s(cnt);
  std::vector<VecItem> vi(cnt);
  for (int i = 0; i < cnt; ++i) {
    lam_s[i] = e.lam[order[i]];
    sig_s[i] = v.sig[order[i]];
    root_s[i] = e.root[order[i]];
    vi[i] = VecItem{e.vec_off[order[i]], (int64_t)i * p->n, p->n, 0};
  }
  CHK(copy_out(lambda, lam_s.data(), cnt * sizeof(double2)));
  if (sigma_min) CHK(copy_out(sigma_min, sig_s.data(), cnt * sizeof(double)));
  if (region_of) CHK(copy_out(region_of, root_s.data(), cnt * sizeof(int32_t)));
  if (vecs && cnt > 0) {
    // permute the gathered vectors into the sorted order on the device, one copy out
    Workspace& ws = p->ws;
    CU(ws.gperm.ensure((size_t)cnt * p->n * sizeof(double2)));
    CU(ws.gitems.ensure(cnt * sizeof(VecItem)));
    CU(cudaMemcpyAsync(ws.gitems.p, vi.data(), cnt * sizeof(VecItem), cudaMemcpyHostToDevice, c.s));
    for (int q0 = 0; q0 < cnt; q0 += 65535) {
      const int k = std::min(65535, cnt - q0);
      prof_begin(PMCIM_K_GATHER, c.s);
      CU(launch_gather_vecs(ws.gdst.as<double2>(), ws.gperm.as<double2>(), ws.gitems.as<VecItem>() + q0, k, p->n,
                            c.s));
      prof_end(PMCIM_K_GATHER, c.s);
    }
    CU(cudaStreamSynchronize(c.s));
    CHK(copy_out(vecs, ws.gperm.p, (size_t)cnt * p->n * sizeof(double2)));
  }
  return PMCIM_OK;
}

int pmcim_batch_solve(int32_t P, const pmcim_batch_item* items, const pmcim_options* opt, int32_t cap,
                      double* lambda, double* sigma_min, int32_t* problem_of, int32_t* region_of, int32_t* count,
                      pmcim_stats* stats) {
  CHK(check_options(opt));
  if (P < 1 || !items) return fail(PMCIM_EINVAL, "empty batch");
  if (!count || cap < 0 || (cap > 0 && !lambda)) return fail(PMCIM_EINVAL, "bad output arguments");
  Call c;
  c.opt = opt;
  if (!items[0].problem) return fail(PMCIM_EINVAL, "batch item 0: problem is NULL");
  c.ws = &items[0].problem->ws;
  CHK(call_stream(*c.ws, opt, &c.s));
  std::vector<HostRegion> top;
  std::vector<int> root_base(P);
  for (int q = 0; q < P; ++q) {
    const pmcim_batch_item& it = items[q];
    if (!it.problem) return fail(PMCIM_EINVAL, "batch item %d: problem is NULL", q);
    CHK(check_regions(it.R, it.regions, it.l));
    CHK(upload_V(it.problem, it.l, it.V, c.s));
    c.groups.push_back(Group{it.problem, it.l, PMCIM_PREC_FP64});
    root_base[q] = (int)top.size();
    std::vector<HostRegion> h = to_host_regions(it.R, it.regions, q, (int)top.size());
    top.insert(top.end(), h.begin(), h.end());
  }
  {
    // each problem's probe block lives in its handle: a handle may appear once per batch
    std::vector<pmcim_problem> hs;
    for (int q = 0; q < P; ++q) hs.push_back(items[q].problem);
    std::sort(hs.begin(), hs.end());
    if (std::adjacent_find(hs.begin(), hs.end()) != hs.end())
      return fail(PMCIM_EINVAL, "a problem handle appears twice in one batch");
  }
  CHK(upload_problems(c));
  EigOut e;
  Verified v;
  std::vector<int> rstat;
  CHK(run_pmcimb(c, top, &e, &v, &rstat, nullptr));
  std::vector<int> order;
  for (size_t i = 0; i < e.lam.size(); ++i)
    if (v.acc[i]) order.push_back((int)i);
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (e.prob[a] != e.prob[b]) return e.prob[a] < e.prob[b];
    if (e.lam[a].x != e.lam[b].x) return e.lam[a].x < e.lam[b].x;
    return e.lam[a].y < e.lam[b].y;
  });
  const int cnt = (int)order.size();
  CHK(copy_out(count, &cnt, sizeof(int32_t)));
  if (stats) CHK(copy_out(stats, &c.st, sizeof(c.st)));
  if (cnt > cap) return fail(PMCIM_ECAPACITY, "%d eigenvalues exceed capacity %d", cnt, cap);
  std::vector<double2> lam_s(cnt);
  std::vector<double> sig_s(cnt);
  std::vector<int32_t> prob_s(cnt), reg_s(cnt);
  for (int i = 0; i < cnt; ++i) {
    const int k = order[i];
    lam_s[i] = e.lam[k];
    sig_s[i] = v.sig[k];
    prob_s[i] = e.prob[k];
    reg_s[i] = e.root[k] - root_base[e.prob[k]];
  }
  CHK(copy_out(lambda, lam_s.data(), cnt * sizeof(double2)));
  if (sigma_min) CHK(copy_out(sigma_min, sig_s.data(), cnt * sizeof(double)));
  if (problem_of) CHK(copy_out(problem_of, prob_s.data(), cnt * sizeof(int32_t)));
  if (region_of) CHK(copy_out(region_of, reg_s.data(), cnt * sizeof(int32_t)));
  return PMCIM_OK;
}

int pmcim_screen_features(pmcim_problem p, const pmcim_options* opt, int32_t R, const pmcim_region* reg,
                          int32_t l, const double* V, double* ind3, float* feats) {
  if (!p) return fail(PMCIM_EINVAL, "problem is NULL");
  CHK(check_options(opt));
  CHK(check_regions(R, reg, l));
  for (int g = 0; g < R; ++g)
    if (reg[g].N % 16) return fail(PMCIM_EINVAL, "region %d: N = %d is not a multiple of 16", g, reg[g].N);
  Call c;
  CHK(single_call(c, p, opt, l, V));
  LevelOut lo;
  CHK(run_level(c, to_host_regions(R, reg, 0), false, false, &lo, nullptr, true));
  CU(cudaStreamSynchronize(c.s));
  if (ind3) CHK(copy_out(ind3, p->ws.ind3.p, (size_t)R * 3 * sizeof(double)));
  if (feats) CHK(copy_out(feats, p->ws.feats.p, (size_t)R * 3 * sizeof(float)));
  return PMCIM_OK;
}

namespace {
struct TmpBuf {
  void* p = nullptr;
  ~TmpBuf() {
    if (p) cudaFree(p);
  }
};
}  // namespace

int pmcim_screen_train(int32_t M, const float* feats, const uint8_t* labels, int32_t epochs, int32_t batch,
                       double lr, double pos_weight, float* params, double* epoch_loss, void* cuda_stream) {
  if (M < 1 || epochs < 0 || batch < 1 || !feats || !labels || !params || !(lr > 0.0) || !(pos_weight > 0.0))
    return fail(PMCIM_EINVAL, "bad training arguments");
  CHK(check_device());
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int B = std::min(batch, M);
  TmpBuf f, y, w, el, sc;
  CU(cudaMalloc(&f.p, (size_t)M * 3 * sizeof(float)));
  CU(cudaMalloc(&y.p, (size_t)M));
  CU(cudaMalloc(&w.p, PMCIM_SCREEN_PARAMS * sizeof(float)));
  CU(cudaMalloc(&el.p, std::max(1, epochs) * sizeof(double)));
  CU(cudaMalloc(&sc.p, screen_train_scratch_bytes(B)));
  CU(cudaMemcpyAsync(f.p, feats, (size_t)M * 3 * sizeof(float), cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(y.p, labels, (size_t)M, cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(w.p, params, PMCIM_SCREEN_PARAMS * sizeof(float), cudaMemcpyDefault, s));
  prof_begin(PMCIM_K_SCREEN, s);
  CU(screen_train(M, (const float*)f.p, (const uint8_t*)y.p, epochs, B, (float)lr, (float)pos_weight, (float*)w.p,
                  (double*)el.p, sc.p, s));
  prof_end(PMCIM_K_SCREEN, s);
  CU(cudaMemcpyAsync(params, w.p, PMCIM_SCREEN_PARAMS * sizeof(float), cudaMemcpyDefault, s));
  if (epoch_loss && epochs > 0) CU(cudaMemcpyAsync(epoch_loss, el.p, epochs * sizeof(double), cudaMemcpyDefault, s));
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

int pmcim_screen_apply(int32_t M, const float* feats, const float* params, float* prob, void* cuda_stream) {
  if (M < 0 || (M > 0 && (!feats || !params || !prob))) return fail(PMCIM_EINVAL, "bad arguments");
  if (M == 0) return PMCIM_OK;
  CHK(check_device());
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  TmpBuf f, w, pr, sc;
  CU(cudaMalloc(&f.p, (size_t)M * 3 * sizeof(float)));
  CU(cudaMalloc(&w.p, PMCIM_SCREEN_PARAMS * sizeof(float)));
  CU(cudaMalloc(&pr.p, (size_t)M * sizeof(float)));
  CU(cudaMalloc(&sc.p, 2 * PMCIM_SCREEN_PARAMS + 256));
  CU(cudaMemcpyAsync(f.p, feats, (size_t)M * 3 * sizeof(float), cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(w.p, params, PMCIM_SCREEN_PARAMS * sizeof(float), cudaMemcpyDefault, s));
  prof_begin(PMCIM_K_SCREEN, s);
  CU(screen_forward(M, (const float*)f.p, (const float*)w.p, (float*)pr.p, sc.p, s));
  prof_end(PMCIM_K_SCREEN, s);
  CU(cudaMemcpyAsync(prob, pr.p, (size_t)M * sizeof(float), cudaMemcpyDefault, s));
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

int pmcim_screen_gradient(int32_t M, const float* feats, const uint8_t* labels, double pos_weight,
                          const float* params, float* grad, double* loss, void* cuda_stream) {
  if (M < 1 || !feats || !labels || !params || !grad || !(pos_weight > 0.0)) return fail(PMCIM_EINVAL, "bad arguments");
  CHK(check_device());
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  TmpBuf f, y, w, g, l, sc;
  CU(cudaMalloc(&f.p, (size_t)M * 3 * sizeof(float)));
  CU(cudaMalloc(&y.p, (size_t)M));
  CU(cudaMalloc(&w.p, PMCIM_SCREEN_PARAMS * sizeof(float)));
  CU(cudaMalloc(&g.p, PMCIM_SCREEN_PARAMS * sizeof(float)));
  CU(cudaMalloc(&l.p, sizeof(double)));
  CU(cudaMalloc(&sc.p, screen_grad_scratch_bytes(M)));
  CU(cudaMemcpyAsync(f.p, feats, (size_t)M * 3 * sizeof(float), cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(y.p, labels, (size_t)M, cudaMemcpyDefault, s));
  CU(cudaMemcpyAsync(w.p, params, PMCIM_SCREEN_PARAMS * sizeof(float), cudaMemcpyDefault, s));
  prof_begin(PMCIM_K_SCREEN, s);
  CU(screen_gradient(M, (const float*)f.p, (const uint8_t*)y.p, (float)pos_weight, (const float*)w.p, (float*)g.p,
                     (double*)l.p, sc.p, s));
  prof_end(PMCIM_K_SCREEN, s);
  CU(cudaMemcpyAsync(grad, g.p, PMCIM_SCREEN_PARAMS * sizeof(float), cudaMemcpyDefault, s));
  if (loss) CU(cudaMemcpyAsync(loss, l.p, sizeof(double), cudaMemcpyDefault, s));
  CU(cudaStreamSynchronize(s));
  return PMCIM_OK;
}

int pmcim_debug_wait_limits(int64_t tc_wait_cycles, int64_t handoff_wait_cycles) {
  if (tc_wait_cycles < 0 || handoff_wait_cycles < 0) return fail(PMCIM_EINVAL, "negative wait limit");
  std::lock_guard<std::mutex> g(g_wait_mu);
  g_tc_wait = tc_wait_cycles ? (long long)tc_wait_cycles : kTcWaitCycles;
  g_handoff_wait = handoff_wait_cycles ? (long long)handoff_wait_cycles : kHandoffWaitCycles;
  return PMCIM_OK;
}

}  // extern "C"
