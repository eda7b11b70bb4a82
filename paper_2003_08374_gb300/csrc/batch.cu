// batch.cu -- host-side plan of a batch of domains: the block tables that map
// every launch's flat block index to (domain, local block), and the device
// tables of per-domain views.  Built once per batch composition.
#include <algorithm>
#include <vector>

#include "mdbs_internal.cuh"

namespace mdbs {

namespace {

long long items_of(long long n, int rep) { return (n + (long long)kBlock * rep - 1) / ((long long)kBlock * rep); }

long long faces_total(const Prm& P) { return P.nf[0] + P.nf[1] + (P.dim == 3 ? P.nf[2] : 0); }

}  // namespace

cudaError_t plan_create(const StepDom* sd, const CgDom* cg, int ndom, int flexible, int smooth_rows, int snake,
                        int sweep_kz, int tail_ctas, int coarse_coop, int vec_sweeps, BatchPlan* out) {
  BatchPlan B{};
  B.ndom = ndom;
  B.flexible = flexible;
  B.snake = snake;
  B.sweep_kz = sweep_kz;
  B.tail_ctas = tail_ctas;
  B.coarse_coop = coarse_coop;
  B.vec_sweeps = vec_sweeps;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // grids cover every work item (one item per block) up to 64 waves of resident
  // blocks; larger spaces loop (grid stride)
  B.grid_cap = sms * (2048 / kBlock) * 64;
  {
    cudaError_t e = sweep_kernel_setup();
    if (e != cudaSuccess) return e;
  }
  // host block tables: spaces in a fixed order, each ndom + 1 prefix entries
  const int nspace = 5 + 6 * kMaxLevels;
  std::vector<int> tab((size_t)nspace * (ndom + 1), 0);
  auto fill = [&](int space, auto count) -> int {
    int* t = &tab[(size_t)space * (ndom + 1)];
    long long acc = 0;
    for (int d = 0; d < ndom; d++) {
      t[d] = (int)acc;
      acc += count(d);
    }
    t[ndom] = (int)acc;
    return (int)acc;
  };
  int totals[5 + 6 * kMaxLevels];
  // one row of kBlock elements per item, except the reduction spaces (kRepBig rows:
  // fewer block reductions and partials)
  int reps[5 + 6 * kMaxLevels];
  for (int q = 0; q < 5 + 6 * kMaxLevels; q++) reps[q] = 1;
  reps[3] = reps[4] = kRepBig;
  reps[5 + kMaxLevels] = smooth_rows;  // finest-level red/black half sweeps
  auto blocks_of = [&](long long n, int space) { return items_of(n, reps[space]); };
  totals[0] = fill(0, [&](int d) { return blocks_of(sd[d].P.cells, 0); });
  totals[1] = fill(1, [&](int d) { return blocks_of(faces_total(sd[d].P), 1); });
  totals[2] = fill(2, [&](int) { return 1LL; });
  totals[3] = fill(3, [&](int d) { return blocks_of(sd[d].P.cells, 3); });
  totals[4] = fill(4, [&](int d) { return blocks_of(faces_total(sd[d].P), 4); });
  B.max_first = 0;
  B.max_levels = 0;
  B.any_cfl = 0;
  B.tail_words = 0;
  for (int d = 0; d < ndom; d++) {
    long long words = 0;
    for (int l = cg[d].first; l < cg[d].nlev; l++) {
      const Level<double>& L = cg[d].ld[l];
      words += 2LL * L.n[0] * L.n[1] * L.n[2];
    }
    B.tail_words = std::max(B.tail_words, words);
    B.max_first = std::max(B.max_first, cg[d].first);
    B.max_levels = std::max(B.max_levels, cg[d].nlev);
    if (sd[d].P.cfl > 0.0) B.any_cfl = 1;
  }
  for (int l = 0; l < kMaxLevels; l++) {
    auto cells_at = [&](int d, int lev) -> long long {
      const Level<double>& L = cg[d].ld[lev];
      return (long long)L.n[0] * L.n[1] * L.n[2];
    };
    const int s0 = 5 + l, s1 = 5 + kMaxLevels + l, s2 = 5 + 2 * kMaxLevels + l, s3 = 5 + 3 * kMaxLevels + l;
    totals[s0] = fill(s0, [&](int d) { return l < cg[d].nlev ? blocks_of(cells_at(d, l), s0) : 0LL; });
    totals[s1] = fill(s1, [&](int d) -> long long {
      if (l >= cg[d].first) return 0;
      const Level<double>& L = cg[d].ld[l];
      return blocks_of((long long)((L.n[0] + 1) / 2) * L.n[1] * L.n[2], s1);
    });
    totals[s2] = fill(s2, [&](int d) { return l < cg[d].first ? blocks_of(cells_at(d, l), s2) : 0LL; });
    totals[s3] = fill(s3, [&](int d) { return l < cg[d].first ? blocks_of(cells_at(d, l + 1), s3) : 0LL; });
    // vector half sweeps: every domain whose level l precedes its tail needs n_x a
    // multiple of 2 V (aligned colour runs) and, in FP32, coefficients that are not BF16
    const int V = flexible ? 4 : 2;
    bool vec_ok = true;
    for (int d = 0; d < ndom; d++) {
      if (l >= cg[d].first) continue;
      if (cg[d].ld[l].n[0] % (2 * V) != 0) vec_ok = false;
      if (flexible && cg[d].lf[l].Tb[0] != nullptr) vec_ok = false;
    }
    if (vec_ok) B.vec_levels |= 1u << l;
    const int s5 = 5 + 5 * kMaxLevels + l;
    totals[s5] = fill(s5, [&](int d) -> long long {
      if (!vec_ok || l >= cg[d].first) return 0;
      const Level<double>& L = cg[d].ld[l];
      const long long halfs = (long long)(L.n[0] / 2) * L.n[1] * L.n[2];
      return (halfs / V + kBlock - 1) / kBlock;
    });
    const int s4 = 5 + 4 * kMaxLevels + l;
    totals[s4] = fill(s4, [&](int d) -> long long {
      if (l >= cg[d].first || sweep_kz <= 0) return 0;
      const Level<double>& L = cg[d].ld[l];
      return (long long)((L.n[0] + kSweepTX - 1) / kSweepTX) * ((L.n[1] + kSweepTY - 1) / kSweepTY) *
             ((L.n[2] + sweep_kz - 1) / sweep_kz);
    });
  }
  cudaError_t e = cudaMalloc(&B.table_storage, tab.size() * sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(B.table_storage, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&B.sd, ndom * sizeof(StepDom));
  if (e == cudaSuccess) e = cudaMemcpy(B.sd, sd, ndom * sizeof(StepDom), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&B.cg, ndom * sizeof(CgDom));
  if (e == cudaSuccess) e = cudaMemcpy(B.cg, cg, ndom * sizeof(CgDom), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&B.any_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B.err_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(B.err_flag, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B.coop_ctr, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(B.coop_ctr, 0, sizeof(unsigned long long));
  if (e == cudaSuccess && coarse_coop) e = coop_grid_size(flexible, B.tail_words, &B.coop_grid);
  if (e != cudaSuccess) {
    plan_destroy(&B);
    return e;
  }
  auto work = [&](int space) {
    Work w;
    w.blk = B.table_storage + (size_t)space * (ndom + 1);
    w.ndom = ndom;
    w.total = totals[space];
    w.rep = reps[space];
    return w;
  };
  B.cells = work(0);
  B.faces = work(1);
  B.dom = work(2);
  B.rcells = work(3);
  B.rfaces = work(4);
  for (int l = 0; l < kMaxLevels; l++) {
    B.lcells[l] = work(5 + l);
    B.lhalf[l] = work(5 + kMaxLevels + l);
    B.lfine[l] = work(5 + 2 * kMaxLevels + l);
    B.lcoarse[l] = work(5 + 3 * kMaxLevels + l);
    B.lsweep[l] = work(5 + 4 * kMaxLevels + l);
    B.lvec[l] = work(5 + 5 * kMaxLevels + l);
  }
  *out = B;
  return cudaSuccess;
}

void plan_destroy(BatchPlan* B) {
  if (B->table_storage) cudaFree(B->table_storage);
  if (B->sd) cudaFree(B->sd);
  if (B->cg) cudaFree(B->cg);
  if (B->any_flag) cudaFree(B->any_flag);
  if (B->err_flag) cudaFree(B->err_flag);
  if (B->coop_ctr) cudaFree(B->coop_ctr);
  B->coop_ctr = nullptr;
  B->table_storage = nullptr;
  B->sd = nullptr;
  B->cg = nullptr;
  B->any_flag = nullptr;
  B->err_flag = nullptr;
}

}  // namespace mdbs
