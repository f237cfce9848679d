// engine.cu -- descriptors and work lists for a set of configurations evaluated together.
//
// A member keeps its own device buffers (Ctx).  The engine uploads one CfgDev per member, the member lists
// of each precision, and the work items of the twiddle kernel and of the two persistent hot kernels.  Items
// of the hot kernels are ordered by estimated cost, largest first, so that the dynamic queue ends with small
// items (longest-processing-time order).  A member's launch shape (particle splits, column splits, staging
// chunk) depends on that member alone, so its arithmetic, and its result, is the same in every batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <numeric>

#include "ssh_internal.h"

namespace ssh {

CfgDev make_cfgdev(const Ctx* c, bool fire_mode) {
  CfgDev g;
  memset(&g, 0, sizeof g);
  g.d = c->d;
  g.nrows = (int)c->tl.rows.size();
  g.lo_base = c->tl.lo_base;
  g.hi_base = c->tl.hi_base;
  g.qmin = c->tl.qmin;
  g.ksplit = c->launch[0].f_ksplit;
  g.nblk = c->n_red_blocks;
  g.N = c->N;
  g.M = c->M;
  g.Npad = c->Npad;
  for (int p = 0; p < 3; p++) {
    const Launch& L = c->launch[p];
    int64_t plen = (c->N + L.nt_psplit - 1) / L.nt_psplit;
    plen = (plen + L.nt_pchunk - 1) / L.nt_pchunk * L.nt_pchunk;
    g.plen[p] = plen;
    g.psplit[p] = (int)((c->N + plen - 1) / plen);
    g.pchunk[p] = L.nt_pchunk;
  }
  g.s_hi = (double*)c->s_hi.p;
  g.s_lo = (double*)c->s_lo.p;
  g.rows = (const TabRow*)c->rows.p;
  g.slots = (const NtSlot*)c->slots.p;
  g.blocks = (const NtBlock*)c->blocks.p;
  g.g_rows = (const int32_t*)c->grows.p;
  g.wk = (const double*)c->wk.p;
  g.cols = (const FCol*)c->cols.p;
  g.fsplit = (const int32_t*)c->fsplit.p;
  g.tab = c->tab.p;
  g.part = c->part.p;
  g.C_hi = (double*)c->C_hi.p;
  g.C_lo = (double*)c->C_lo.p;
  g.S_hi = (double*)c->S_hi.p;
  g.S_lo = (double*)c->S_lo.p;
  g.coef = c->coef.p;
  g.blk = c->blk.p;
  g.scal = (double*)c->scal.p;
  g.fpart = c->fpart.p;
  g.F_hi = (double*)c->F_hi.p;
  g.F_lo = (double*)c->F_lo.p;
  g.pref = c->pref;
  g.inv_L = c->inv_L;
  g.L = c->L;
  tc_fill_cfgdev(c, &g);
  if (c->fire) fire_fill_cfgdev(c, &g);
  if (!fire_mode) g.run = nullptr;
  return g;
}

void engine_free(Engine* e) {
  for (DevBuf* b : {&e->d_cfgs, &e->d_lists, &e->d_tw, &e->d_nt, &e->d_f, &e->d_counters, &e->d_tclist, &e->d_tcprep,
                    &e->d_tcdens, &e->d_tcforce, &e->d_bm}) {
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->bytes = 0;
  }
}

static cudaError_t up(DevBuf* b, const void* src, size_t bytes, cudaStream_t st) {
  if (b->p && b->bytes < bytes) {
    cudaFree(b->p);
    b->p = nullptr;
  }
  if (!b->p) {
    b->bytes = std::max<size_t>(bytes, 16);
    cudaError_t e = cudaMalloc(&b->p, b->bytes);
    if (e != cudaSuccess) return e;
  }
  if (bytes == 0) return cudaSuccess;
  return cudaMemcpyAsync(b->p, src, bytes, cudaMemcpyHostToDevice, st);
}

cudaError_t engine_build(Engine* e, const std::vector<Ctx*>& members, const std::vector<int>& prec_of, bool fire_mode,
                         cudaStream_t st) {
  e->members = members;
  e->prec_of = prec_of;
  e->fire_mode = fire_mode;
  const int n = (int)members.size();
  if (n > 0) {
    e->device = members[0]->device;
    e->sm_count = members[0]->sm_count;
  }
  e->host_cfgs.resize(n);
  for (int i = 0; i < n; i++) e->host_cfgs[i] = make_cfgdev(members[i], fire_mode);
  // member lists: one per precision, then all members
  std::vector<int> lists[3];
  for (int i = 0; i < n; i++)
    for (int p = 0; p < 3; p++)
      if (prec_of[i] == p || prec_of[i] < 0) lists[p].push_back(i);
  e->h_lists.clear();
  int off[4];
  for (int p = 0; p < 3; p++) {
    off[p] = (int)e->h_lists.size();
    e->h_lists.insert(e->h_lists.end(), lists[p].begin(), lists[p].end());
  }
  off[3] = (int)e->h_lists.size();
  for (int i = 0; i < n; i++) e->h_lists.push_back(i);
  // work items per precision
  e->h_tw.clear();
  e->h_nt.clear();
  e->h_f.clear();
  int tw_off[3], nt_off[3], f_off[3], tw_n[3], nt_n[3], f_n[3];
  for (int p = 0; p < 3; p++) {
    tw_off[p] = (int)e->h_tw.size();
    nt_off[p] = (int)e->h_nt.size();
    f_off[p] = (int)e->h_f.size();
    std::vector<std::pair<double, NtItem>> nt;
    std::vector<std::pair<double, FItem>> fi;
    for (int i : lists[p]) {
      const Ctx* c = members[i];
      const CfgDev& g = e->host_cfgs[i];
      if (p == SSH_FX && c->tc.on) continue;  // tensor-core members have their own work lists
      const int64_t total = (int64_t)g.nrows * g.Npad;
      for (int64_t s = 0; s < total; s += kTwThreads) e->h_tw.push_back({i, 0, s});
      for (int b = 0; b < (int)c->nt.blocks.size(); b++)
        for (int ps = 0; ps < g.psplit[p]; ps++) {
          const int64_t j0 = ps * g.plen[p], j1 = std::min(c->N, j0 + g.plen[p]);
          nt.push_back({(double)c->nt.blocks[b].nslots * (double)(j1 - j0), {i, b, ps, 0}});
        }
      const int pblocks = (int)((c->N + kForceThreads - 1) / kForceThreads);
      for (int ks = 0; ks < g.ksplit; ks++) {
        const int c0 = c->f_split[ks], c1 = c->f_split[ks + 1];
        const int64_t k0 = c0 < (int)c->fp.cols.size() ? c->fp.cols[c0].k0 : c->M;
        const int64_t k1 = c1 < (int)c->fp.cols.size() ? c->fp.cols[c1].k0 : c->M;
        for (int pb = 0; pb < pblocks; pb++) fi.push_back({(double)(k1 - k0 + (c1 - c0)), {i, pb, ks, 0}});
      }
    }
    // largest first; ties keep their construction order (stable), so the list is deterministic
    std::stable_sort(nt.begin(), nt.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::stable_sort(fi.begin(), fi.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (auto& x : nt) e->h_nt.push_back(x.second);
    for (auto& x : fi) e->h_f.push_back(x.second);
    tw_n[p] = (int)e->h_tw.size() - tw_off[p];
    nt_n[p] = (int)e->h_nt.size() - nt_off[p];
    f_n[p] = (int)e->h_f.size() - f_off[p];
  }
  // tensor-core members (fixed point), in particle-chunk phases: phase ph holds chunk ph of every member that has
  // one; chunks after the first get descriptors of their own, after the members'
  std::vector<int> tcl;
  std::vector<TwItem> tcp;
  std::vector<TcItem> tcd, tcf;
  int64_t tc_grid = 0;
  size_t tc_smem = 0;
  int64_t tc_nd = 0;
  int nph = 0;
  for (int i : lists[SSH_FX])
    if (members[i]->tc.on) {
      tcl.push_back(i);
      nph = std::max(nph, tc_chunks(members[i]));
      tc_grid = std::max<int64_t>(tc_grid, (int64_t)(members[i]->tc.R1 + 1) * members[i]->tc.nP);
      tc_smem = std::max(tc_smem, members[i]->tc.prep_smem);
      tc_nd = std::max<int64_t>(tc_nd, (int64_t)members[i]->tc.d * members[i]->N);
    }
  if (nph > kMaxTcPhases) return cudaErrorInvalidValue;
  std::vector<std::vector<int>> ccfg(n);  // [member][chunk] -> descriptor index
  for (int i : tcl) {
    ccfg[i].assign(tc_chunks(members[i]), i);
    for (int ch = 1; ch < (int)ccfg[i].size(); ch++) {
      CfgDev g = e->host_cfgs[i];
      tc_chunk_cfgdev(members[i], ch, &g);
      ccfg[i][ch] = (int)e->host_cfgs.size();
      e->host_cfgs.push_back(g);
    }
  }
  TcPhase phs[kMaxTcPhases];
  std::vector<std::vector<BlockMap>> tab_bm(nph), rtab_bm(nph);
  // largest first over all members of a phase (the persistent GEMM takes items from a queue in list order):
  // density items one by one; force items by bundle (the column tiles of one particle tile, kept together so that
  // they share its digits in L2), bundles by their total K-steps (a stable sort keeps each bundle contiguous and
  // in order)
  auto by_size = [](const TcItem& a, const TcItem& b) { return a.nks > b.nks; };
  for (int ph = 0; ph < nph; ph++) {
    TcPhase& P = phs[ph];
    int64_t steps = 0;  // density K-steps of the phase: each member gets its share of the SMs
    for (int i : tcl)
      if (tc_chunks(members[i]) > ph) steps += tc_density_steps(members[i], ph);
    P.prep_off = (int)tcp.size();
    P.dens_off = (int)tcd.size();
    P.force_off = (int)tcf.size();
    // preparation items of the four-axis members last (they run on their own instance of the kernel)
    for (int four = 0; four < 2; four++)
      for (int i : tcl)
        if (tc_chunks(members[i]) > ph && (members[i]->tc.d == 4) == (four == 1)) {
          const size_t before = tcp.size();
          tc_prep_items(members[i], ccfg[i][ph], ph, tcp);
          if (four) P.prep4 += (int)(tcp.size() - before);
        }
    for (int i : tcl) {
      if (tc_chunks(members[i]) <= ph) continue;
      const int cfg = ccfg[i][ph];
      for (int64_t b = 0; b < tc_table_blocks(members[i], ph); b++) tab_bm[ph].push_back({cfg, (int32_t)b});
      const int64_t share = (int64_t)((double)e->sm_count * (double)tc_density_steps(members[i], ph) /
                                      (double)std::max<int64_t>(1, steps) * (double)e->tune.dens_pct / 100.0);
      tc_gemm_items(members[i], cfg, ph, share, tcd, tcf);
    }
    P.prep_n = (int)tcp.size() - P.prep_off;
    P.dens_n = (int)tcd.size() - P.dens_off;
    P.force_n = (int)tcf.size() - P.force_off;
    std::stable_sort(tcd.begin() + P.dens_off, tcd.end(), by_size);
    if (e->tune.force_bundle) {
      std::map<std::pair<int, int>, int64_t> bundle;
      for (size_t k = P.force_off; k < tcf.size(); k++) bundle[{tcf[k].cfg, tcf[k].a}] += tcf[k].nks;
      std::stable_sort(tcf.begin() + P.force_off, tcf.end(), [&](const TcItem& a, const TcItem& b) {
        return bundle[{a.cfg, a.a}] > bundle[{b.cfg, b.a}];
      });
      // the last items of the queue decide when the launch ends: the final two items per SM go largest first, so the
      // launch ends on the shortest ones
      const size_t tail = std::min<size_t>(tcf.size() - P.force_off, 2 * (size_t)e->sm_count);
      std::stable_sort(tcf.end() - tail, tcf.end(), by_size);
    } else {
      std::stable_sort(tcf.begin() + P.force_off, tcf.end(), by_size);
    }
    // before the force items of this chunk: the preparation again for members whose buffers hold a later chunk
    P.rprep_off = (int)tcp.size();
    for (int i : tcl) {
      if (tc_chunks(members[i]) - 1 <= ph) continue;
      for (int64_t b = 0; b < tc_table_blocks(members[i], ph); b++) rtab_bm[ph].push_back({ccfg[i][ph], (int32_t)b});
    }
    for (int four = 0; four < 2; four++)
      for (int i : tcl)
        if (tc_chunks(members[i]) - 1 > ph && (members[i]->tc.d == 4) == (four == 1)) {
          const size_t before = tcp.size();
          tc_prep_items(members[i], ccfg[i][ph], ph, tcp);
          if (four) P.rprep4 += (int)(tcp.size() - before);
        }
    P.rprep_n = (int)tcp.size() - P.rprep_off;
  }
  cudaError_t err;
  if ((err = up(&e->d_tclist, tcl.data(), sizeof(int) * tcl.size(), st)) != cudaSuccess) return err;
  if ((err = up(&e->d_tcprep, tcp.data(), sizeof(TwItem) * tcp.size(), st)) != cudaSuccess) return err;
  if ((err = up(&e->d_tcdens, tcd.data(), sizeof(TcItem) * tcd.size(), st)) != cudaSuccess) return err;
  if ((err = up(&e->d_tcforce, tcf.data(), sizeof(TcItem) * tcf.size(), st)) != cudaSuccess) return err;
  // block maps: only the blocks each member needs
  std::vector<BlockMap> bm;
  auto add_blocks = [&](int cfg, int64_t nb) {
    for (int64_t b = 0; b < nb; b++) bm.push_back({cfg, (int32_t)b});
  };
  size_t bm_off[6], bm_n[6];
  bm_off[0] = bm.size();
  for (int i = 0; i < n; i++) add_blocks(i, e->host_cfgs[i].nb_fire);
  bm_n[0] = bm.size() - bm_off[0];
  bm_off[1] = bm.size();
  for (int i = 0; i < n; i++) add_blocks(i, ((int64_t)members[i]->d * members[i]->N + 63) / 64);
  bm_n[1] = bm.size() - bm_off[1];
  bm_off[2] = bm.size();  // tables, phase by phase
  for (int ph = 0; ph < nph; ph++) {
    phs[ph].tab_off = (int)(bm.size() - bm_off[2]);
    bm.insert(bm.end(), tab_bm[ph].begin(), tab_bm[ph].end());
    phs[ph].tab_n = (int)tab_bm[ph].size();
    phs[ph].rtab_off = (int)(bm.size() - bm_off[2]);
    bm.insert(bm.end(), rtab_bm[ph].begin(), rtab_bm[ph].end());
    phs[ph].rtab_n = (int)rtab_bm[ph].size();
  }
  bm_n[2] = bm.size() - bm_off[2];
  bm_off[3] = bm.size();
  for (int i : tcl) add_blocks(i, tc_finish_blocks(*members[i]));
  bm_n[3] = bm.size() - bm_off[3];
  bm_off[4] = bm.size();
  for (int i : tcl) add_blocks(i, tc_coef_blocks(*members[i]));
  bm_n[4] = bm.size() - bm_off[4];
  bm_off[5] = bm.size();
  for (int i : tcl) add_blocks(i, ((int64_t)members[i]->d * members[i]->N + 63) / 64);
  bm_n[5] = bm.size() - bm_off[5];
  if ((err = up(&e->d_bm, bm.data(), sizeof(BlockMap) * bm.size(), st)) != cudaSuccess) return err;
  const BlockMap* dbm = (const BlockMap*)e->d_bm.p;
  e->bm_dots = dbm + bm_off[0];
  e->nbm_dots = (int)bm_n[0];
  e->bm_nd = dbm + bm_off[1];
  e->nbm_nd = (int)bm_n[1];
  if ((err = up(&e->d_cfgs, e->host_cfgs.data(), sizeof(CfgDev) * e->host_cfgs.size(), st)) != cudaSuccess) return err;
  if ((err = up(&e->d_lists, e->h_lists.data(), sizeof(int) * e->h_lists.size(), st)) != cudaSuccess) return err;
  if ((err = up(&e->d_tw, e->h_tw.data(), sizeof(TwItem) * e->h_tw.size(), st)) != cudaSuccess) return err;
  if ((err = up(&e->d_nt, e->h_nt.data(), sizeof(NtItem) * e->h_nt.size(), st)) != cudaSuccess) return err;
  if ((err = up(&e->d_f, e->h_f.data(), sizeof(FItem) * e->h_f.size(), st)) != cudaSuccess) return err;
  if (!e->d_counters.p) {
    // [0], [1] integer-pipe density and force queues; [2], [3] and [4], [5] tensor-core density and force
    // queues with their finished-CTA counts (reset by the kernels themselves)
    e->d_counters.bytes = 64;
    if ((err = cudaMalloc(&e->d_counters.p, 64)) != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(e->d_counters.p, 0, 64, st)) != cudaSuccess) return err;
  }
  const CfgDev* dc = (const CfgDev*)e->d_cfgs.p;
  const int* dl = (const int*)e->d_lists.p;
  for (int p = 0; p < 3; p++) {
    EngineView& v = e->view[p];
    v = EngineView();
    v.cfgs = dc;
    v.list = dl + off[p];
    v.nlist = (int)lists[p].size();
    v.tw = (const TwItem*)e->d_tw.p + tw_off[p];
    v.ntw = tw_n[p];
    v.nt = (const NtItem*)e->d_nt.p + nt_off[p];
    v.nnt = nt_n[p];
    v.fi = (const FItem*)e->d_f.p + f_off[p];
    v.nfi = f_n[p];
    v.counters = (int*)e->d_counters.p;
    v.sm_count = e->sm_count;
    if (p == SSH_FX) {
      v.tc_list = (const int*)e->d_tclist.p;
      v.ntc_list = (int)tcl.size();
      v.tc_prep = (const TwItem*)e->d_tcprep.p;
      v.ntc_prep = (int)tcp.size();
      v.tc_dens = (const TcItem*)e->d_tcdens.p;
      v.ntc_dens = (int)tcd.size();
      v.tc_force = (const TcItem*)e->d_tcforce.p;
      v.ntc_force = (int)tcf.size();
      v.tc_max_grid = tc_grid;
      v.tc_prep_smem = tc_smem;
      v.tc_maxND = tc_nd;
      v.tc_bm_tab = dbm + bm_off[2];
      v.ntc_bm_tab = (int)bm_n[2];
      v.ntc_phase = nph;
      for (int ph = 0; ph < nph; ph++) v.tc_ph[ph] = phs[ph];
      v.tc_bm_fin = dbm + bm_off[3];
      v.ntc_bm_fin = (int)bm_n[3];
      v.tc_bm_coef = dbm + bm_off[4];
      v.ntc_bm_coef = (int)bm_n[4];
      v.tc_bm_ff = dbm + bm_off[5];
      v.ntc_bm_ff = (int)bm_n[5];
    }
    for (int i : lists[p]) {
      const Ctx* c = members[i];
      v.nt_smem = std::max(v.nt_smem, c->launch[p].nt_smem);
      v.maxM = std::max(v.maxM, c->M);
      v.maxND = std::max(v.maxND, (int64_t)c->d * c->N);
      v.maxblk = std::max(v.maxblk, c->n_red_blocks);
    }
  }
  e->all = dl + off[3];
  e->nall = n;
  e->maxND_all = 0;
  e->max_nb_fire = 0;
  for (int i = 0; i < n; i++) {
    e->maxND_all = std::max(e->maxND_all, (int64_t)members[i]->d * members[i]->N);
    e->max_nb_fire = std::max(e->max_nb_fire, e->host_cfgs[i].nb_fire);
  }
  return cudaGetLastError();
}

}  // namespace ssh
