// Host side of the discrete adjoint (include/lbpwfa.h: lbpwfa_record,
// lbpwfa_adjoint_step): the recording window, its checkpoints or tape, and
// the reverse sweep that queues the kernels of lb_adjoint.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lb_adjoint_types.cuh"
#include "lb_adjoint_dispatch.h"
#include "lb_runtime.h"

using namespace lbp;

namespace lbprt {

constexpr int kRowSets = 64;  // reverse steps per gradient flush

struct AdjRec {
  AdjKernelSet ak{};
  bool armed = false;
  long long start_step = 0, len = 0, cap = 0, C = 0;
  // checkpoints: the forward writes the tape of the window's last two
  // segments (from step pre_from on) into their halves, so the sweep
  // recomputes neither when the window was stepped to its end; -1: none
  long long pre_from = -1;
  bool start_from_driver = false;
  int start_have_prev = 0;
  size_t entry_bytes = 0;   // one tape entry
  size_t state_bytes = 0;   // one checkpoint: f, E, B, prev
  Buf tape, ckpt, prev0, finalst;
  std::vector<int> ckpt_have_prev;
  Buf lf[2], lE[2], lB[2], lp[2], rA, rG, rEn, rBn, cA, cF, cU, lAf, cW;
  Buf rows, setp, gpart, g3, gp, Tx, Kx, jv;
  int ntx = 1;
  size_t bytes = 0;
  // checkpoints: the next segment is recomputed on a second stream while
  // this one is reversed; each has its own half of the tape
  cudaStream_t rs = nullptr;
  cudaEvent_t ev_rec[2] = {nullptr, nullptr};  // tape half filled
  cudaEvent_t ev_rev[2] = {nullptr, nullptr};  // tape half consumed
};

namespace {

void free_rec(lbpwfa_s* h, AdjRec* r) {
  Buf* all[] = {&r->tape, &r->ckpt, &r->prev0, &r->finalst, &r->lf[0], &r->lf[1], &r->lE[0], &r->lE[1],
                &r->lB[0], &r->lB[1], &r->lp[0], &r->lp[1], &r->rA, &r->rG, &r->rEn, &r->rBn, &r->cA,
                &r->cF, &r->cU, &r->lAf, &r->cW, &r->rows,
                &r->setp, &r->gpart, &r->g3, &r->gp, &r->Tx, &r->Kx, &r->jv};
  for (Buf* b : all) {
    h->device_bytes -= b->bytes;
    release(*b);
  }
  for (int j = 0; j < 2; ++j) {
    if (r->ev_rec[j]) cudaEventDestroy(r->ev_rec[j]);
    if (r->ev_rev[j]) cudaEventDestroy(r->ev_rev[j]);
    r->ev_rec[j] = r->ev_rev[j] = nullptr;
  }
  if (r->rs) cudaStreamDestroy(r->rs);
  r->rs = nullptr;
}

int ab(lbpwfa_s* h, AdjRec* r, Buf& b, size_t bytes) {
  int st = alloc(h, b, bytes);
  if (st == LBPWFA_OK) r->bytes += bytes;
  return st;
}

// copy the current state (f, E, B, prev) to / from a checkpoint slot
int save_state(lbpwfa_s* h, char* dst) {
  const size_t pb = h->f[0].bytes, fb = h->E[0].bytes;
  CK(h, cudaMemcpyAsync(dst, h->f[h->cur].p, pb, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dst + pb, h->E[h->cur].p, fb, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(dst + pb + fb, h->B[h->cur].p, fb, cudaMemcpyDeviceToDevice, h->stream));
  if (h->prev.bytes)
    CK(h, cudaMemcpyAsync(dst + pb + 2 * fb, h->prev.p, h->prev.bytes, cudaMemcpyDeviceToDevice, h->stream));
  return LBPWFA_OK;
}
int restore_state(lbpwfa_s* h, const char* src) {
  const size_t pb = h->f[0].bytes, fb = h->E[0].bytes;
  CK(h, cudaMemcpyAsync(h->f[h->cur].p, src, pb, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->E[h->cur].p, src + pb, fb, cudaMemcpyDeviceToDevice, h->stream));
  CK(h, cudaMemcpyAsync(h->B[h->cur].p, src + pb + fb, fb, cudaMemcpyDeviceToDevice, h->stream));
  if (h->prev.bytes)
    CK(h, cudaMemcpyAsync(h->prev.p, src + pb + 2 * fb, h->prev.bytes, cudaMemcpyDeviceToDevice, h->stream));
  return LBPWFA_OK;
}

}  // namespace

int adj_before_step(lbpwfa_s* h, void** tape) {
  *tape = nullptr;
  AdjRec* r = h->adj;
  if (!r || !r->armed) return LBPWFA_OK;
  if (r->len >= r->cap) {
    h->err = "lbpwfa_step: the recording window is full (lbpwfa_record max_steps)";
    return LBPWFA_ERR_STATE;
  }
  if (r->C == 0) {
    *tape = (char*)r->tape.p + (size_t)r->len * r->entry_bytes;
  } else {
    const long long s = r->len / r->C;
    if (r->len % r->C == 0) {
      int st = save_state(h, (char*)r->ckpt.p + (size_t)s * r->state_bytes);
      if (st != LBPWFA_OK) return st;
      r->ckpt_have_prev[s] = h->have_prev;
    }
    if (r->pre_from >= 0 && r->len >= r->pre_from)
      *tape = (char*)r->tape.p + ((size_t)(s & 1) * r->C + (size_t)(r->len - s * r->C)) * r->entry_bytes;
  }
  r->len += 1;
  return LBPWFA_OK;
}

void adj_invalidate(lbpwfa_s* h) {
  if (h->adj) {
    h->adj->armed = false;
    h->adj->len = 0;
  }
}

void adj_free(lbpwfa_s* h) {
  if (!h->adj) return;
  free_rec(h, h->adj);
  delete h->adj;
  h->adj = nullptr;
}

}  // namespace lbprt

using namespace lbprt;

extern "C" int lbpwfa_record(lbpwfa_t h, const lbpwfa_record_params* rp) {
  if (!h || !rp) return LBPWFA_ERR_INVALID;
  if (h->in_batch || h->prm.dim > 2 || h->prm.precision == LBPWFA_FP16S || h->prm.geometry != LBPWFA_CARTESIAN) {
    h->err = "lbpwfa_record: the adjoint covers single Cartesian 1D/2D runs with FP64 or FP32 storage";
    return LBPWFA_ERR_INVALID;
  }
  if (rp->max_steps < 1 || rp->checkpoint_every < 0) return LBPWFA_ERR_INVALID;
  CK(h, cudaStreamSynchronize(h->stream));
  adj_free(h);
  AdjRec* r = new AdjRec();
  h->adj = r;
  // exact-sum FP32 storage reverses with the FP32 kernels (the same real type)
  const int adj_prec = h->prm.precision == LBPWFA_FP32C ? LBPWFA_FP32 : h->prm.precision;
  if (!adjoint_kernels(h->prm.dim, h->prm.closure, adj_prec, &r->ak)) {
    adj_free(h);
    return LBPWFA_ERR_INVALID;
  }
  {
    // the kernels address the planes of a tape entry, of the per-set
    // velocity terms (K x dim) and of a population set with 32-bit offsets
    const long long span = std::max({(long long)r->ak.NTAPE, (long long)r->ak.K * h->prm.dim, (long long)h->Q});
    if (span * h->plane >= (1LL << 31)) {
      adj_free(h);
      h->err = "lbpwfa_record: " + std::to_string(span) + " planes of " + std::to_string(h->plane) +
               " cells pass 32-bit offsets";
      return LBPWFA_ERR_INVALID;
    }
  }
  r->cap = rp->max_steps;
  r->C = rp->checkpoint_every >= rp->max_steps ? 0 : rp->checkpoint_every;
  const size_t rs = h->real_sz, pl = (size_t)h->plane;
  r->entry_bytes = (size_t)r->ak.NTAPE * pl * rs;
  r->state_bytes = h->f[0].bytes + 2 * h->E[0].bytes + h->prev.bytes;
  r->ntx = h->prm.dim == 2 ? (h->n[1] + r->ak.tx - 1) / r->ak.tx : 1;
  int st = LBPWFA_OK;
  if (r->C == 0) {
    st = ab(h, r, r->tape, (size_t)r->cap * r->entry_bytes);
    if (st == LBPWFA_OK && h->prev.bytes) st = ab(h, r, r->prev0, h->prev.bytes);
  } else {
    const long long nck = (r->cap + r->C - 1) / r->C;
    r->pre_from = (nck >= 2 ? nck - 2 : 0) * r->C;
    st = ab(h, r, r->tape, 2 * (size_t)r->C * r->entry_bytes);
    if (st == LBPWFA_OK) st = ab(h, r, r->ckpt, (size_t)nck * r->state_bytes);
    if (st == LBPWFA_OK) st = ab(h, r, r->finalst, r->state_bytes);
    r->ckpt_have_prev.assign((size_t)nck, 0);
    cudaError_t e = cudaStreamCreateWithFlags(&r->rs, cudaStreamNonBlocking);
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
      e = cudaEventCreateWithFlags(&r->ev_rec[j], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_rev[j], cudaEventDisableTiming);
    }
    if (st == LBPWFA_OK && e != cudaSuccess) st = fail_cuda(h, e, "lbpwfa_record: recompute stream");
  }
  const size_t popb = (size_t)h->K * h->Q * pl * rs, fldb = 3 * pl * rs;
  for (int j = 0; j < 2 && st == LBPWFA_OK; ++j) {
    st = ab(h, r, r->lf[j], popb);
    if (st == LBPWFA_OK) st = ab(h, r, r->lE[j], fldb);
    if (st == LBPWFA_OK) st = ab(h, r, r->lB[j], fldb);
    if (st == LBPWFA_OK && r->ak.NPREV) st = ab(h, r, r->lp[j], (size_t)r->ak.NPREV * pl * rs);
  }
  if (st == LBPWFA_OK) st = ab(h, r, r->rA, (size_t)r->ak.K * pl * rs);
  if (st == LBPWFA_OK) st = ab(h, r, r->rG, (size_t)r->ak.NG * pl * rs);
  if (st == LBPWFA_OK) st = ab(h, r, r->cA, (size_t)r->ak.K * pl * rs);
  if (st == LBPWFA_OK) st = ab(h, r, r->cF, (size_t)r->ak.K * pl * rs);
  if (st == LBPWFA_OK) st = ab(h, r, r->cU, (size_t)r->ak.K * h->prm.dim * pl * rs);
  if (st == LBPWFA_OK) st = ab(h, r, r->lAf, (size_t)r->ak.K * pl * rs);
  if (st == LBPWFA_OK && h->prm.closure == LBPWFA_WARMC)
    st = ab(h, r, r->cW, 2 * (size_t)h->prm.dim * pl * rs);
  if (st == LBPWFA_OK) st = ab(h, r, r->rEn, fldb);
  if (st == LBPWFA_OK) st = ab(h, r, r->rBn, fldb);
  if (st == LBPWFA_OK) st = ab(h, r, r->rows, (size_t)kRowSets * 2 * r->ntx * h->n[0] * sizeof(double));
  if (st == LBPWFA_OK) st = ab(h, r, r->setp, (size_t)kRowSets * sizeof(double2));
  if (st == LBPWFA_OK) st = ab(h, r, r->gpart, (size_t)kRowSets * 3 * sizeof(double));
  if (st == LBPWFA_OK) st = ab(h, r, r->g3, 4 * sizeof(double));
  if (st == LBPWFA_OK)
    st = ab(h, r, r->gp, (h->profile_h.empty() ? 1 : h->profile_h.size()) * sizeof(double));
  if (st == LBPWFA_OK) st = ab(h, r, r->Tx, 2 * (size_t)h->n[1] * sizeof(double));
  if (st == LBPWFA_OK) st = ab(h, r, r->Kx, 2 * (size_t)h->n[1] * sizeof(double));
  if (st == LBPWFA_OK) st = ab(h, r, r->jv, sizeof(double));
  if (st != LBPWFA_OK) {
    adj_free(h);
    return st;
  }
  // driver transverse factors at the E_z slots, and the initial-field
  // profile k(x) = sigma_r sqrt(pi/2) erf(x / sqrt(2) sigma_r) with its
  // sigma_r derivative (2D)
  {
    const int nx = h->n[1];
    std::vector<double> T(2 * (size_t)nx), Kx(2 * (size_t)nx);
    const double sr = h->prm.sigma_r, dx = h->prm.dx, xoff = 0.5 * (nx - 1);
    for (int i = 0; i < nx; ++i) {
      if (h->prm.dim == 1) {
        T[i] = 1.0;
        T[nx + i] = 0.0;
        Kx[i] = Kx[nx + i] = 0.0;
        continue;
      }
      const double xs = (i - xoff + 0.5) * dx;
      const double t = std::exp(-xs * xs / (2.0 * sr * sr));
      T[i] = t;
      T[nx + i] = t * xs * xs / (sr * sr * sr);
      const double xn = (i - xoff) * dx;
      const double er = std::erf(xn / (std::sqrt(2.0) * sr));
      Kx[i] = -sr * std::sqrt(M_PI / 2.0) * er;
      Kx[nx + i] = -(std::sqrt(M_PI / 2.0) * er - xn / sr * std::exp(-xn * xn / (2.0 * sr * sr)));
    }
    CK(h, cudaMemcpyAsync(r->Tx.p, T.data(), T.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(r->Kx.p, Kx.data(), Kx.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
  }
  if (r->C == 0 && h->prev.bytes)
    CK(h, cudaMemcpyAsync(r->prev0.p, h->prev.p, h->prev.bytes, cudaMemcpyDeviceToDevice, h->stream));
  r->start_step = h->step;
  r->start_have_prev = h->have_prev;
  r->start_from_driver = h->fields_from_driver && h->step == 0 && h->prm.dim == 2;
  r->len = 0;
  r->armed = true;
  return LBPWFA_OK;
}

namespace {

struct Sweep {
  lbpwfa_s* h;
  AdjRec* r;
  int cl = 0;  // adjoint buffers holding the current adjoint state
  int nsets = 0;
  std::vector<double2> setp;

  GradParams grad_params() const {
    GradParams G{};
    G.n0 = h->n[0];
    G.nsets = nsets;
    G.ntx = r->ntx;
    G.rows = (const double*)r->rows.p;
    G.setp = (const double2*)r->setp.p;
    G.dx = h->prm.dx;
    G.alpha = h->prm.alpha;
    G.sigma_z = h->prm.sigma_z;
    G.inv2sz2 = h->prm.sigma_z > 0 ? 1.0 / (2.0 * h->prm.sigma_z * h->prm.sigma_z) : 0.0;
    G.profile = h->profile_d;
    G.plen = (int)h->profile_h.size();
    G.pdz = h->prm.profile_dz;
    G.gpart = (double*)r->gpart.p;
    G.g3 = (double*)r->g3.p;
    G.gp = (double*)r->gp.p;
    return G;
  }

  int flush() {
    if (nsets == 0) return LBPWFA_OK;
    CK(h, cudaMemcpyAsync(r->setp.p, setp.data(), (size_t)nsets * sizeof(double2), cudaMemcpyHostToDevice,
                          h->stream));
    launch_grad(grad_params(), h->stream);
    CK_LAUNCH(h, "adjoint gradient kernels");
    // the host copy of the set table is reused by the next flush
    CK(h, cudaStreamSynchronize(h->stream));
    nsets = 0;
    return LBPWFA_OK;
  }

  double* rows_of_set(int j) const {
    return (double*)r->rows.p + (size_t)j * 2 * r->ntx * h->n[0];
  }

  // reverse step of window step j; `entry` is its tape entry, `entry_prev`
  // the previous step's (or null, then `prev0` holds the values it read)
  int reverse(long long j, const void* entry, const void* entry_prev, const void* prev0, bool first) {
    AdjParams A{};
    A.P = step_params(h);
    A.P.have_prev = j > 0 ? (h->NPREV ? 1 : 0) : r->start_have_prev;
    A.tape = entry;
    A.tape_prev = entry_prev;
    A.prev0 = prev0;
    A.lf_in = r->lf[cl].p;
    A.lf_out = r->lf[1 - cl].p;
    A.lE_in = r->lE[cl].p;
    A.lE_out = r->lE[1 - cl].p;
    A.lB_in = r->lB[cl].p;
    A.lB_out = r->lB[1 - cl].p;
    A.lp_in = first ? nullptr : r->lp[cl].p;
    A.lp_out = r->lp[1 - cl].p;
    A.rA = r->rA.p;
    A.rG = r->rG.p;
    A.rEn = r->rEn.p;
    A.rBn = r->rBn.p;
    A.cA = r->cA.p;
    A.cF = r->cF.p;
    A.cU = r->cU.p;
    A.lAf = r->lAf.p;
    A.cW = r->cW.p;
    A.rows = rows_of_set(nsets);
    A.Tx = (const double*)r->Tx.p;
    const dim3 g((unsigned)((h->n[0] + r->ak.tz - 1) / r->ak.tz), (unsigned)r->ntx, 1);
    // 2D: extra block rows for the edge band (see adj_coll_kernel)
    A.band_rows = 0;
    if (h->prm.dim == 2 && h->n[0] >= 7 && h->n[1] >= 7) {
      const long long band = 6LL * h->n[0] + 6LL * (h->n[1] - 6);
      const long long per_row = (long long)g.x * r->ak.tz * r->ak.tx;
      A.band_rows = (int)((band + per_row - 1) / per_row);
    }
    const dim3 gk(g.x, g.y + (unsigned)A.band_rows, (unsigned)((r->ak.K + r->ak.spt - 1) / r->ak.spt));
    r->ak.coll(A, gk, h->stream);
    CK_LAUNCH(h, "adj_coll_kernel launch");
    r->ak.local(A, g, h->stream);
    CK_LAUNCH(h, "adj_local_kernel launch");
    r->ak.field(A, g, h->stream);
    CK_LAUNCH(h, "adj_field_kernel launch");
    setp.push_back(make_double2(zeta0_of(h->prm.z0, r->start_step + j, h->dt), 0.0));
    nsets += 1;
    cl = 1 - cl;
    if (nsets == kRowSets) {
      int st = flush();
      setp.clear();
      if (st != LBPWFA_OK) return st;
    }
    return LBPWFA_OK;
  }
};

}  // namespace

extern "C" int lbpwfa_adjoint_step(lbpwfa_t h, lbpwfa_adjoint_io* io) {
  if (!h || !io) return LBPWFA_ERR_INVALID;
  AdjRec* r = h->adj;
  if (!r || !r->armed || r->len < 1) {
    h->err = "lbpwfa_adjoint_step: no recorded steps (call lbpwfa_record, then lbpwfa_step)";
    return LBPWFA_ERR_STATE;
  }
  const int wz = io->witness[0], wx = h->prm.dim >= 2 ? io->witness[1] : 0;
  if (wz < 0 || wz >= h->n[0] || wx < 0 || wx >= h->n[1]) return LBPWFA_ERR_INVALID;
  const long long wid = (long long)wz + (long long)wx * h->nzp;

  // J and the seed
  r->ak.read_slot(h->E[h->cur].p, lo_of(h, h->E[h->cur]), wid, (double*)r->jv.p, h->stream);
  CK_LAUNCH(h, "read_slot_kernel launch");
  for (int j = 0; j < 2; ++j) {
    CK(h, cudaMemsetAsync(r->lf[j].p, 0, r->lf[j].bytes, h->stream));
    CK(h, cudaMemsetAsync(r->lE[j].p, 0, r->lE[j].bytes, h->stream));
    CK(h, cudaMemsetAsync(r->lB[j].p, 0, r->lB[j].bytes, h->stream));
    if (r->lp[j].p) CK(h, cudaMemsetAsync(r->lp[j].p, 0, r->lp[j].bytes, h->stream));
  }
  CK(h, cudaMemsetAsync(r->rBn.p, 0, r->rBn.bytes, h->stream));
  // the first reverse step forms the next state's population adjoints from
  // zero gathered values and zero lambda_A
  CK(h, cudaMemsetAsync(r->lAf.p, 0, r->lAf.bytes, h->stream));
  CK(h, cudaMemsetAsync(r->g3.p, 0, r->g3.bytes, h->stream));
  CK(h, cudaMemsetAsync(r->gp.p, 0, r->gp.bytes, h->stream));
  r->ak.seed(r->lE[0].p, wid, io->seed, h->stream);
  CK_LAUNCH(h, "adj_seed_kernel launch");

  Sweep S{h, r};
  S.setp.reserve(kRowSets);
  const long long end_step = h->step;
  const int end_cur = h->cur, end_have_prev = h->have_prev;
  bool first = true;
  if (r->C == 0) {
    for (long long j = r->len - 1; j >= 0; --j) {
      const char* e = (const char*)r->tape.p + (size_t)j * r->entry_bytes;
      int st = S.reverse(j, e, j > 0 ? e - r->entry_bytes : nullptr, j > 0 ? nullptr : r->prev0.p, first);
      if (st != LBPWFA_OK) return st;
      first = false;
    }
  } else {
    int st = save_state(h, (char*)r->finalst.p);
    if (st != LBPWFA_OK) return st;
    const long long nseg = (r->len + r->C - 1) / r->C;
    // segments from pre_seg on hold the tape the forward wrote (the window
    // was stepped to its end); the halves are overwritten below, so a retry
    // after an error recomputes every segment
    const long long pre_seg = r->pre_from >= 0 && r->len == r->cap ? r->pre_from / r->C : nseg;
    r->pre_from = -1;
    // segment s is recomputed into tape half s % 2 on the second stream, as
    // soon as the reverse of segment s + 2 has consumed that half, so the
    // recompute of segment s - 1 runs while segment s is reversed
    cudaStream_t ms = h->stream;
    auto half = [&](long long s) { return (char*)r->tape.p + (size_t)(s & 1) * r->C * r->entry_bytes; };
    for (int j = 0; j < 2; ++j) CK(h, cudaEventRecord(r->ev_rev[j], ms));  // after the state was saved
    for (long long s = pre_seg; s < nseg; ++s) CK(h, cudaEventRecord(r->ev_rec[s & 1], ms));  // written in order
    auto recompute = [&](long long s) -> int {
      const long long b = s * r->C, e = std::min(r->len, b + r->C);
      CK(h, cudaStreamWaitEvent(r->rs, r->ev_rev[s & 1], 0));
      h->stream = r->rs;
      int rc = restore_state(h, (const char*)r->ckpt.p + (size_t)s * r->state_bytes);
      h->step = r->start_step + b;
      h->have_prev = r->ckpt_have_prev[s];
      for (long long j = b; j < e && rc == LBPWFA_OK; ++j) rc = launch_step(h, half(s) + (size_t)(j - b) * r->entry_bytes);
      h->stream = ms;
      if (rc != LBPWFA_OK) return rc;
      CK(h, cudaEventRecord(r->ev_rec[s & 1], r->rs));
      return LBPWFA_OK;
    };
    if (nseg - 1 < pre_seg) {
      st = recompute(nseg - 1);
      if (st != LBPWFA_OK) return st;
    }
    for (long long s = nseg - 1; s >= 0; --s) {
      const long long b = s * r->C, e = std::min(r->len, b + r->C);
      CK(h, cudaStreamWaitEvent(ms, r->ev_rec[s & 1], 0));
      if (s > 0 && s - 1 < pre_seg) {
        st = recompute(s - 1);
        if (st != LBPWFA_OK) return st;
      }
      const char* ck = (const char*)r->ckpt.p + (size_t)s * r->state_bytes;
      const char* prev_ck = h->prev.bytes ? ck + h->f[0].bytes + 2 * h->E[0].bytes : nullptr;
      for (long long j = e - 1; j >= b; --j) {
        const char* en = half(s) + (size_t)(j - b) * r->entry_bytes;
        st = S.reverse(j, en, j > b ? en - r->entry_bytes : nullptr, j > b ? nullptr : prev_ck, first);
        if (st != LBPWFA_OK) return st;
        first = false;
      }
      CK(h, cudaEventRecord(r->ev_rev[s & 1], ms));
    }
  }
  int st = S.flush();
  if (st != LBPWFA_OK) return st;
  S.setp.clear();
  // the driver's initial fields (2D, window from step 0)
  if (r->start_from_driver && r->start_step == 0) {
    StepParams P = step_params(h);
    const dim3 g((unsigned)((h->n[0] + r->ak.tz - 1) / r->ak.tz), (unsigned)r->ntx, 1);
    r->ak.init_rows(P, r->lE[S.cl].p, r->lB[S.cl].p, (const double*)r->Kx.p, S.rows_of_set(0), g, h->stream);
    CK_LAUNCH(h, "adj_init_rows_kernel launch");
    S.setp.push_back(make_double2(h->prm.z0 - 0.5 * h->dt, 0.5 * h->prm.dx));
    S.setp.push_back(make_double2(h->prm.z0, 0.0));
    S.nsets = 2;
    st = S.flush();
    if (st != LBPWFA_OK) return st;
  }
  double g4[4] = {0, 0, 0, 0}, J = 0.0;
  CK(h, cudaMemcpyAsync(g4, r->g3.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaMemcpyAsync(&J, r->jv.p, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (io->grad_profile && !h->profile_h.empty())
    CK(h, cudaMemcpyAsync(io->grad_profile, r->gp.p, h->profile_h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
  h->step = end_step;
  h->cur = end_cur;
  h->have_prev = end_have_prev;
  if (r->C != 0) {
    st = restore_state(h, (const char*)r->finalst.p);
    if (st != LBPWFA_OK) return st;
  }
  CK(h, cudaStreamSynchronize(h->stream));
  for (int q = 0; q < 3; ++q) io->grad_driver[q] = g4[q];
  io->J = J;
  r->armed = false;
  r->len = 0;
  return LBPWFA_OK;
}
