// Batched chi0 over many q-points and frequencies: resident pair elements, persistent
// contraction launches over job tables, CUDA-graph capture per call signature, autotuning.
#include "api_internal.h"

namespace gwapi {
// ------------------------------------------------------------------ batched path (many q, many w)
// Every requested slot's M is produced once and kept resident; the contraction of all
// (q, w) blocks then runs as one persistent launch (FP64) or one persistent launch per
// frequency over all slots (split precision).  The whole sequence is captured once per
// call signature into a CUDA graph and replayed.  Launch shapes come from a small
// autotuner that times the candidates on the first call of a signature.
struct BatchLayout {
    std::vector<int64_t> P, moff, doff, coff, dgoff;
    std::vector<int> ng;
    // split precision: pair segments of at most pair_chunk pairs, each with its own
    // column exponents and slices (the exactness bound of the slice sums is per segment)
    struct Seg {
        int q;
        int64_t p0, cnt, kpad, zoff, eoff;
    };
    std::vector<Seg> seg;
    size_t Mtot = 0, Dtot = 0, Ztot = 0, Etot = 0;
};

BatchLayout batch_layout(gw_chi0 *h, int nq, const int *iq, int nw)
{
    BatchLayout L;
    size_t coff = 0, dgoff = 0;
    const int64_t kseg = h->d.pair_chunk;
    for (int i = 0; i < nq; ++i) {
        const int ng = h->sph[iq[i]].ng;
        const int64_t P = (int64_t)h->val[iq[i]].nb * h->cond.nb;
        L.ng.push_back(ng);
        L.P.push_back(P);
        L.moff.push_back((int64_t)L.Mtot);
        L.doff.push_back((int64_t)L.Dtot);
        L.coff.push_back((int64_t)coff);
        L.dgoff.push_back((int64_t)dgoff);
        L.Mtot += (size_t)P * ng;
        L.Dtot += (size_t)nw * P;
        coff += (size_t)nw * ng * ng;
        dgoff += (size_t)nw * ng;
        for (int64_t p0 = 0; p0 < P; p0 += kseg) {
            BatchLayout::Seg sg;
            sg.q = i;
            sg.p0 = p0;
            sg.cnt = std::min(kseg, P - p0);
            sg.kpad = (sg.cnt + 63) / 64 * 64;
            sg.zoff = (int64_t)L.Ztot;
            sg.eoff = (int64_t)L.Etot;
            L.Ztot += (size_t)h->d.nslices * 2 * ng * sg.kpad;
            L.Etot += (size_t)ng;
            L.seg.push_back(sg);
        }
    }
    return L;
}

std::string batch_key(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, const void *chi,
                      const void *diag)
{
    std::string k = "p" + std::to_string(h->d.prec) + "s" + std::to_string(h->d.nslices) + "m" +
                    std::to_string(h->d.mtxel_prec) + "|";
    char buf[64];
    for (int i = 0; i < nq; ++i) k += std::to_string(iq[i]) + ":" + std::to_string(h->sph[iq[i]].ng) + ",";
    k += "|";
    for (int i = 0; i < nw; ++i) {
        snprintf(buf, sizeof buf, "%a,", omega[i]);
        k += buf;
    }
    snprintf(buf, sizeof buf, "|%p|%p", chi, diag);
    return k + buf;
}

std::string tune_key(gw_chi0 *h, const BatchLayout &L, int nw)
{
    std::string k = "p" + std::to_string(h->d.prec) + "s" + std::to_string(h->d.nslices) + "w" + std::to_string(nw);
    for (size_t i = 0; i < L.ng.size(); ++i) k += "," + std::to_string(L.ng[i]) + "x" + std::to_string(L.P[i]);
    return k;
}

// Enqueue the producer stages: pair elements of every slot, Delta, and (split precision)
// the square roots.  The slices depend on the frequency and are enqueued per frequency.
gw_status batch_stage_a(gw_chi0 *h, int nq, const int *iq, const gw::OmegaList &om, const BatchLayout &L)
{
    for (int i = 0; i < nq; ++i) {
        const BandSet &v = h->val[iq[i]];
        gw::PairPlan pp = pair_plan(h, h->sph[iq[i]]);
        {
            Scope sc(h, "pair_mtxel");
            CK(h, run_pair(h, v.psi, h->cond.psi, h->cond.nb, 0, L.P[i], pp, h->Mall + L.moff[i]), "pair kernel");
        }
        Scope sc(h, "delta");
        CK(h, gw::launch_delta(v.energy, h->cond.energy, h->cond.nb, 0, L.P[i], om, h->Dall + L.doff[i], h->st),
           "delta");
    }
    if (h->d.prec == GW_PREC_OZAKI_BF16) {
        Scope sc(h, "oz_split");
        CK(h, gw::launch_oz_sqrt(h->Dall, (int64_t)L.Dtot, h->SPall, h->st), "oz sqrt");
    }
    return GW_OK;
}

gw_status batch_oz_split(gw_chi0 *h, int nq, int w, const BatchLayout &L)
{
    (void)nq;
    Scope sc(h, "oz_split");
    for (const auto &sg : L.seg) {
        const int ng = L.ng[sg.q];
        const double *sp = h->SPall + L.doff[sg.q] + (int64_t)w * L.P[sg.q] + sg.p0;
        const double2 *M = h->Mall + L.moff[sg.q] + sg.p0 * ng;
        CK(h, gw::launch_oz_colexp(M, sg.cnt, ng, sp, h->Eall + sg.eoff, h->st), "oz exponents");
        CK(h, gw::launch_oz_slice(M, sg.cnt, ng, sp, h->Eall + sg.eoff, h->d.nslices, sg.kpad,
                                  (uint16_t *)h->Zall + sg.zoff, h->st),
           "oz slices");
    }
    return GW_OK;
}

gw_status batch_f64_jobs(gw_chi0 *h, int nq, int nw, const BatchLayout &L, double2 *chi, int bt,
                         std::vector<gw::F64Job> &jobs)
{
    jobs.clear();
    for (int i = 0; i < nq; ++i) {
        gw_status s = f64_jobs(h, jobs, h->Mall + L.moff[i], L.P[i], L.ng[i], h->Dall + L.doff[i], L.P[i], nw,
                               chi + L.coff[i], bt);
        if (s) return s;
    }
    return GW_OK;
}

gw_status batch_oz_jobs(gw_chi0 *h, int nq, int w, const BatchLayout &L, double2 *chi, int bn,
                        std::vector<gw::OzJob> &jobs)
{
    (void)nq;
    jobs.clear();
    for (const auto &sg : L.seg) {
        const int ng = L.ng[sg.q];
        gw::OzJob j;
        gw_status s = oz_job(h, j, (uint16_t *)h->Zall + sg.zoff, sg.kpad, ng, h->Eall + sg.eoff,
                             chi + L.coff[sg.q] + (int64_t)w * ng * ng, bn);
        if (s) return s;
        jobs.push_back(j);
    }
    return GW_OK;
}

// Time each launch-shape candidate of the contraction on the real data (into chi, which
// is cleared afterwards by the real run) and keep the fastest.
gw_status batch_autotune(gw_chi0 *h, int nq, const int *iq, int nw, const gw::OmegaList &om, const BatchLayout &L,
                         double2 *chi)
{
    const std::string key = tune_key(h, L, nw);
    auto it = h->tune_cache.find(key);
    if (it != h->tune_cache.end()) {
        h->tuned_bt = it->second[0];
        h->tuned_waves = it->second[1];
        h->tuned_bn = it->second[2];
        h->bn_tuned = h->d.prec != GW_PREC_FP64;
        return GW_OK;
    }
    gw_status s = batch_stage_a(h, nq, iq, om, L);
    if (s) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::array<int, 3> pick = {h->tuned_bt, h->tuned_waves, h->tuned_bn};
    const bool saved_timing = h->timing;
    h->timing = false;
    if (h->d.prec == GW_PREC_FP64) {
        for (int bt : {64, 32})
            for (int waves : {2, 4, 8}) {
                std::vector<gw::F64Job> jobs;
                if ((s = batch_f64_jobs(h, nq, nw, L, chi, bt, jobs))) break;
                cudaEventRecord(e0, h->st);
                if ((s = launch_f64_jobs(h, jobs, bt, waves))) break;
                cudaEventRecord(e1, h->st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    pick = {bt, waves, h->tuned_bn};
                }
            }
    } else if (!(s = batch_oz_split(h, nq, 0, L))) {
        for (int bn : {256, 240, 128}) {
            std::vector<gw::OzJob> jobs;
            if ((s = batch_oz_jobs(h, nq, 0, L, chi, bn, jobs))) break;
            cudaEventRecord(e0, h->st);
            if ((s = launch_oz_jobs(h, jobs, bn))) break;
            cudaEventRecord(e1, h->st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                pick = {h->tuned_bt, h->tuned_waves, bn};
            }
        }
    }
    h->timing = saved_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    h->tune_cache[key] = pick;
    h->tuned_bt = pick[0];
    h->tuned_waves = pick[1];
    h->tuned_bn = pick[2];
    h->bn_tuned = h->d.prec != GW_PREC_FP64;
    return GW_OK;
}

gw_status compute_batch(gw_chi0 *h, int nq, const int *iq, int nw, const double *omega, const gw::OmegaList &om,
                        double *chi, double *diag)
{
    const BatchLayout L = batch_layout(h, nq, iq, nw);
    gw_status s;
    if ((s = grow(h, (void **)&h->Mall, &h->Mall_cap, sizeof(double2) * L.Mtot, "resident M")) ||
        (s = grow(h, (void **)&h->Dall, &h->Dall_cap, sizeof(double) * L.Dtot, "resident Delta")))
        return s;
    if (h->d.prec == GW_PREC_OZAKI_BF16 &&
        ((s = grow(h, (void **)&h->SPall, &h->SPall_cap, sizeof(double) * L.Dtot, "resident scales")) ||
         (s = grow(h, &h->Zall, &h->Zall_cap, sizeof(uint16_t) * L.Ztot, "resident slices")) ||
         (s = grow(h, (void **)&h->Eall, &h->Eall_cap, sizeof(int) * L.Etot, "resident exponents"))))
        return s;
    if (!h->cap_st) CK(h, cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking), "capture stream");
    if ((s = batch_autotune(h, nq, iq, nw, om, L, (double2 *)chi))) return s;

    const std::string key = batch_key(h, nq, iq, nw, omega, chi, diag) + "|" + std::to_string(h->tuned_bt) + "," +
                            std::to_string(h->tuned_waves) + "," + std::to_string(h->tuned_bn);
    gw_chi0::Graph *g = nullptr;
    for (auto &x : h->graphs)
        if (x.key == key) g = &x;
    if (!g) {
        // job tables first (outside the capture), in a buffer owned by the graph
        std::vector<gw::F64Job> fj;
        std::vector<std::vector<gw::OzJob>> oj(nw);
        std::vector<unsigned char> blob;
        std::vector<size_t> offs;
        if (h->d.prec == GW_PREC_FP64) {
            if ((s = batch_f64_jobs(h, nq, nw, L, (double2 *)chi, h->tuned_bt, fj))) return s;
            f64_schedule(fj, h->tuned_waves);
            offs.push_back(0);
            blob.resize(sizeof(gw::F64Job) * fj.size());
            std::memcpy(blob.data(), fj.data(), blob.size());
        } else {
            for (int w = 0; w < nw; ++w) {
                if ((s = batch_oz_jobs(h, nq, w, L, (double2 *)chi, h->tuned_bn, oj[w]))) return s;
                oz_schedule(oj[w]);
                offs.push_back(blob.size());
                blob.resize(blob.size() + sizeof(gw::OzJob) * oj[w].size());
                std::memcpy(blob.data() + offs.back(), oj[w].data(), sizeof(gw::OzJob) * oj[w].size());
            }
        }
        gw_chi0::Graph ng;
        ng.key = key;
        ng.jobs_bytes = blob.size();
        if ((s = dalloc(h, &ng.jobs, ng.jobs_bytes, "graph job tables"))) return s;
        CK(h, cudaMemcpy(ng.jobs, blob.data(), blob.size(), cudaMemcpyHostToDevice), "graph job tables");

        cudaStream_t user = h->st;
        const bool saved_timing = h->timing;
        h->timing = false;
        h->st = h->cap_st;
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
        gw_status body = GW_OK;
        if (ce == cudaSuccess) {
            for (int i = 0; i < nq && !body; ++i) {
                if (cudaMemsetAsync((double2 *)chi + L.coff[i], 0, sizeof(double2) * (size_t)nw * L.ng[i] * L.ng[i],
                                    h->st) != cudaSuccess ||
                    (diag && cudaMemsetAsync(diag + L.dgoff[i], 0, sizeof(double) * (size_t)nw * L.ng[i], h->st) !=
                                 cudaSuccess))
                    body = fail(h, GW_ERR_CUDA, "capture: memset");
            }
            if (!body) body = batch_stage_a(h, nq, iq, om, L);
            if (!body && h->d.prec == GW_PREC_FP64) {
                int nitems = 0;
                for (auto &j : fj) nitems = std::max(nitems, j.item_start + (int)((int64_t)j.ksplit * j.ntile *
                                                                                   (j.ntile + 1) / 2));
                const int grid = std::max(1, std::min(nitems, 2 * num_sms()));
                if (gw::launch_contract_f64_jobs(h->tuned_bt, (const gw::F64Job *)ng.jobs, (int)fj.size(), nitems,
                                                 grid, h->status, h->st) != cudaSuccess)
                    body = fail(h, GW_ERR_CUDA, "capture: contraction");
            } else if (!body) {
                for (int w = 0; w < nw && !body; ++w) {
                    body = batch_oz_split(h, nq, w, L);
                    if (body) break;
                    int nitems = 0;
                    for (auto &j : oj[w]) nitems = std::max(nitems, j.item_start + j.ntiles);
                    const int grid = std::max(1, std::min(nitems, num_sms()));
                    if (gw::launch_oz_gemm_jobs(h->tuned_bn, (const gw::OzJob *)((char *)ng.jobs + offs[w]),
                                                (int)oj[w].size(), nitems, grid, h->status, h->st) != cudaSuccess)
                        body = fail(h, GW_ERR_CUDA, "capture: split contraction");
                }
            }
            for (int i = 0; i < nq && !body; ++i) {
                const double2 *M = h->Mall + L.moff[i];
                if (diag && gw::launch_diag(M, L.P[i], L.ng[i], h->Dall + L.doff[i], L.P[i], nw,
                                            diag + L.dgoff[i], L.ng[i], h->st) != cudaSuccess)
                    body = fail(h, GW_ERR_CUDA, "capture: diag");
                if (!body && gw::launch_symmetrize((double2 *)chi + L.coff[i], L.ng[i], nw, h->st) != cudaSuccess)
                    body = fail(h, GW_ERR_CUDA, "capture: symmetrize");
            }
            ce = cudaStreamEndCapture(h->st, &graph);
        }
        h->st = user;
        h->timing = saved_timing;
        if (body) {
            if (graph) cudaGraphDestroy(graph);
            dfree(h, ng.jobs, ng.jobs_bytes);
            return body;
        }
        if (ce != cudaSuccess) {
            dfree(h, ng.jobs, ng.jobs_bytes);
            return cuda_fail(h, ce, "stream capture");
        }
        ce = cudaGraphInstantiate(&ng.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            dfree(h, ng.jobs, ng.jobs_bytes);
            return cuda_fail(h, ce, "graph instantiate");
        }
        h->graphs.push_back(ng);
        g = &h->graphs.back();
    }
    Scope sc(h, "batch_graph");
    CK(h, cudaGraphLaunch(g->exec, h->st), "graph launch");
    return GW_OK;
}
} // namespace gwapi

