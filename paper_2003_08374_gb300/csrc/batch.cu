// batch.cu -- host-side plan of a batch of domains: the block tables that map
// every launch's flat block index to (domain, local block), and the device
// tables of per-domain views.  Built once per batch composition.
#include <algorithm>
#include <vector>

#include "mdbs_internal.cuh"

namespace mdbs {

namespace {

long long blocks_of(long long n) { return (n + kBlock - 1) / kBlock; }

long long faces_total(const Prm& P) { return P.nf[0] + P.nf[1] + (P.dim == 3 ? P.nf[2] : 0); }

}  // namespace

cudaError_t plan_create(const StepDom* sd, const CgDom* cg, int ndom, int flexible, BatchPlan* out) {
  BatchPlan B{};
  B.ndom = ndom;
  B.flexible = flexible;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  B.grid_cap = sms * (2048 / kBlock);  // one wave of fully resident blocks
  // host block tables: spaces in a fixed order, each ndom + 1 prefix entries
  const int nspace = 3 + 4 * kMaxLevels;
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
  int totals[3 + 4 * kMaxLevels];
  totals[0] = fill(0, [&](int d) { return blocks_of(sd[d].P.cells); });
  totals[1] = fill(1, [&](int d) { return blocks_of(faces_total(sd[d].P)); });
  totals[2] = fill(2, [&](int) { return 1LL; });
  B.max_first = 0;
  B.max_levels = 0;
  B.any_cfl = 0;
  for (int d = 0; d < ndom; d++) {
    B.max_first = std::max(B.max_first, cg[d].first);
    B.max_levels = std::max(B.max_levels, cg[d].nlev);
    if (sd[d].P.cfl > 0.0) B.any_cfl = 1;
  }
  for (int l = 0; l < kMaxLevels; l++) {
    auto cells_at = [&](int d, int lev) -> long long {
      const Level<double>& L = cg[d].ld[lev];
      return (long long)L.n[0] * L.n[1] * L.n[2];
    };
    totals[3 + l] = fill(3 + l, [&](int d) { return l < cg[d].nlev ? blocks_of(cells_at(d, l)) : 0LL; });
    totals[3 + kMaxLevels + l] = fill(3 + kMaxLevels + l, [&](int d) -> long long {
      if (l >= cg[d].first) return 0;
      const Level<double>& L = cg[d].ld[l];
      return blocks_of((long long)((L.n[0] + 1) / 2) * L.n[1] * L.n[2]);
    });
    totals[3 + 2 * kMaxLevels + l] =
        fill(3 + 2 * kMaxLevels + l, [&](int d) { return l < cg[d].first ? blocks_of(cells_at(d, l)) : 0LL; });
    totals[3 + 3 * kMaxLevels + l] =
        fill(3 + 3 * kMaxLevels + l, [&](int d) { return l < cg[d].first ? blocks_of(cells_at(d, l + 1)) : 0LL; });
  }
  cudaError_t e = cudaMalloc(&B.table_storage, tab.size() * sizeof(int));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(B.table_storage, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&B.sd, ndom * sizeof(StepDom));
  if (e == cudaSuccess) e = cudaMemcpy(B.sd, sd, ndom * sizeof(StepDom), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&B.cg, ndom * sizeof(CgDom));
  if (e == cudaSuccess) e = cudaMemcpy(B.cg, cg, ndom * sizeof(CgDom), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&B.any_flag, sizeof(int));
  if (e != cudaSuccess) {
    plan_destroy(&B);
    return e;
  }
  auto work = [&](int space) {
    Work w;
    w.blk = B.table_storage + (size_t)space * (ndom + 1);
    w.ndom = ndom;
    w.total = totals[space];
    return w;
  };
  B.cells = work(0);
  B.faces = work(1);
  B.dom = work(2);
  for (int l = 0; l < kMaxLevels; l++) {
    B.lcells[l] = work(3 + l);
    B.lhalf[l] = work(3 + kMaxLevels + l);
    B.lfine[l] = work(3 + 2 * kMaxLevels + l);
    B.lcoarse[l] = work(3 + 3 * kMaxLevels + l);
  }
  *out = B;
  return cudaSuccess;
}

void plan_destroy(BatchPlan* B) {
  if (B->table_storage) cudaFree(B->table_storage);
  if (B->sd) cudaFree(B->sd);
  if (B->cg) cudaFree(B->cg);
  if (B->any_flag) cudaFree(B->any_flag);
  B->table_storage = nullptr;
  B->sd = nullptr;
  B->cg = nullptr;
  B->any_flag = nullptr;
}

}  // namespace mdbs
