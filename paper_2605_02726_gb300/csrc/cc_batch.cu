// Batched encoder iterations: many images of different sizes, each with its own parameters, Adam
// state and workspace, advance together with ~20 launches per iteration in total instead of ~20
// per image.  A plan (coolchic_batch_create) lays out, in a caller-provided device table, the
// per-job argument structs of every kernel and the CTA range of every job; coolchic_batch_step
// only launches, so it can be captured in a CUDA graph and replayed.
//
// Schedule: for each kernel class the job's CTA count is a fraction of its single-image CTA count
// (never more: the per-CTA partial buffers of the job's workspace are sized for that).  Jobs are
// laid out in the CTA space by decreasing work so that the largest images start first.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/coolchic.h"
#include "cc_kernels.h"

struct cc_batch {
    int n = 0;
    int rd_capacity = 0;
    char* table = nullptr;  // device
    cc::Batch<cc::RelaxArgs> relax;
    cc::Batch<cc::ArmArgs> arm, arm_h;  // jobs without / with hyperlatent grids (two kernel forms)
    cc::Batch<cc::UpFwdArgs> upf[cc::kL];  // index m = 1..5
    cc::Batch<cc::SynArgs> synf, synb;
    cc::Batch<cc::ConvArgs> conv;
    cc::Batch<cc::UpAdjArgs> upa[cc::kL];  // stage 1..6
    cc::Batch<cc::IfceArgs> ifce;
    cc::Batch<cc::GatherArgs> gather;       // last iteration of a call: Adam only
    cc::Batch<cc::GatherArgs> gather_next;  // other iterations: Adam + next step's relaxed latents
    cc::Batch<cc::ReduceArgs> reduce;
    cc::Batch<cc::SoapArgs> soap;  // launched when some job uses CC_OPT_SOAP
    bool any_soap = false;
    cc::Batch<cc::FinishArgs> finish;
    double* rd = nullptr;  // device [rd_capacity][n][3]
};

namespace cc {
namespace {

struct TableWriter {
    std::vector<char> host;
    size_t take(size_t bytes) {
        const size_t o = host.size();
        host.resize(o + ((bytes + 255) & ~(size_t)255), 0);
        return o;
    }
};

// Appends args[order[..]] and the CTA starts; returns the batch descriptor (device pointers
// relative to `dev_base`, fixed up once the table is placed).
template <typename A>
Batch<A> put(TableWriter& tw, const std::vector<A>& args, const std::vector<int>& ctas, const std::vector<int>& order) {
    static_assert(sizeof(A) <= 512, "table_bytes assumes argument structs of at most 512 bytes");
    const int n = (int)order.size();  // the jobs of this table, in CTA order
    const size_t oa = tw.take(sizeof(A) * n), ob = tw.take(sizeof(int) * (n + 1));
    std::vector<int> begin(n + 1, 0);
    for (int q = 0; q < n; ++q) begin[q + 1] = begin[q] + ctas[order[q]];
    for (int q = 0; q < n; ++q) std::memcpy(tw.host.data() + oa + sizeof(A) * q, &args[order[q]], sizeof(A));
    std::memcpy(tw.host.data() + ob, begin.data(), sizeof(int) * (n + 1));
    Batch<A> b;
    b.args = reinterpret_cast<const A*>(oa);  // offsets for now
    b.cta_begin = reinterpret_cast<const int*>(ob);
    b.njobs = n;
    b.total_ctas = begin[n];
    return b;
}

template <typename A>
void place(Batch<A>& b, char* base) {
    b.args = reinterpret_cast<const A*>(base + reinterpret_cast<size_t>(b.args));
    b.cta_begin = reinterpret_cast<const int*>(base + reinterpret_cast<size_t>(b.cta_begin));
}

int scaled(int cap, float f) {
    int c = (int)(cap * f + 0.5f);
    return c < 1 ? 1 : (c > cap ? cap : c);
}

size_t table_bytes(int n, int rd_capacity) {
    // upper bound: 23 kernel tables of at most 512-byte args plus CTA arrays, and the records
    return (size_t)23 * ((size_t)512 * n + 256 + sizeof(int) * (n + 1) + 256) + (size_t)rd_capacity * n * 3 * sizeof(double) + 4096;
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" {

size_t coolchic_batch_table_bytes(int32_t n_jobs, int32_t rd_capacity) {
    if (n_jobs < 1 || rd_capacity < 0) return 0;
    return table_bytes(n_jobs, rd_capacity);
}

}  // extern "C"

namespace cc {
namespace {
// Plans the batch; the table image is uploaded synchronously, or (host_staging non-null) written
// to the pinned host_staging and copied asynchronously on `stream`.
int batch_create_impl(int32_t n, const cc_arch_t* archs, const cc_hparams_t* hps, const float* const* images,
                      const cc_state_t* states, void* const* workspaces, const size_t* ws_bytes,
                      const cc_schedule_t* sched, int32_t rd_capacity, void* table, size_t table_size,
                      void* host_staging, cudaStream_t stream, cc_batch_t** out) {
    if (n < 1 || !archs || !hps || !images || !states || !workspaces || !ws_bytes || !out || rd_capacity < 0)
        return set_error(CC_ERR_ARG, "batch_create: invalid arguments");
    if (!table || ((uintptr_t)table & 255)) return set_error(CC_ERR_WORKSPACE, "batch_create: table NULL or not 256-byte aligned");
    if (table_size < table_bytes(n, rd_capacity)) return set_error(CC_ERR_WORKSPACE, "batch_create: table too small");
    int rc = device_setup_checked();
    if (rc) return rc;
    cc_schedule_t sc = {1.f, 1.f, 1.f, 1.f};
    if (sched) sc = *sched;
    if (!(sc.arm > 0.f && sc.arm <= 1.f && sc.syn > 0.f && sc.syn <= 1.f && sc.conv > 0.f && sc.conv <= 1.f &&
          sc.other > 0.f && sc.other <= 1.f))
        return set_error(CC_ERR_ARG, "batch_create: schedule fractions must lie in (0, 1]");
    std::vector<Work> W(n);
    std::vector<Hp> H(n);
    for (int j = 0; j < n; ++j) {
        cc_arch_t ref;
        if (coolchic_arch_init(&ref, archs[j].H, archs[j].W) != CC_OK) return CC_ERR_ARG;
        ref.hyper_grids = archs[j].hyper_grids;
        if (std::memcmp(&ref, &archs[j], sizeof(ref)) != 0 || (ref.hyper_grids != 0 && ref.hyper_grids != kNH))
            return set_error(CC_ERR_UNSUPPORTED, "batch_create: job %d has an unsupported architecture", j);
        const cc_hparams_t& h = hps[j];
        if (const int rc = validate_hparams(&h)) return rc;
        const cc_state_t& st = states[j];
        if (!images[j] || !st.latents || !st.params || !st.m_lat || !st.v_lat || !st.m_par || !st.v_par || !st.step)
            return set_error(CC_ERR_ARG, "batch_create: job %d has a NULL image or state pointer", j);
        if (h.nn_optimizer == CC_OPT_SOAP && !st.soap)
            return set_error(CC_ERR_ARG, "batch_create: job %d uses CC_OPT_SOAP without a SOAP state", j);
        if (!workspaces[j] || ((uintptr_t)workspaces[j] & 255))
            return set_error(CC_ERR_WORKSPACE, "batch_create: job %d workspace NULL or misaligned", j);
        const size_t need = layout_job(&archs[j], 0, nullptr, nullptr);
        if (ws_bytes[j] < need)
            return set_error(CC_ERR_WORKSPACE, "batch_create: job %d workspace has %zu bytes, needs %zu", j, ws_bytes[j], need);
        layout_job(&archs[j], 0, (char*)workspaces[j], &W[j]);
        W[j].discard_dead = discard_enabled() ? 1 : 0;  // encoder iterations, as in coolchic_encode_step
        H[j] = hp_from(&h);
    }
    // largest jobs first in the CTA space
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return W[x].N > W[y].N; });

    cc_batch* b = new cc_batch();
    b->n = n;
    b->rd_capacity = rd_capacity;
    TableWriter tw;
    std::vector<int> ctas(n);
    auto fill = [&](auto make, auto count) {
        using A = decltype(make(0));
        std::vector<A> args(n);
        for (int j = 0; j < n; ++j) {
            args[j] = make(j);
            ctas[j] = count(j);
        }
        return put(tw, args, ctas, order);
    };
    const size_t rd_off = tw.take((size_t)rd_capacity * n * 3 * sizeof(double) + 8);  // records [slot][job][3]

    // per-job workspace step partial counts follow the schedule
    for (int j = 0; j < n; ++j) {
        Work& w = W[j];
        w.n_cta_arm = scaled(w.n_cta_arm, sc.arm);
        w.n_cta_syn = scaled(w.n_cta_syn, sc.syn);
        w.n_cta_conv = scaled(w.n_cta_conv, sc.conv);
        for (int st = 1; st < kL; ++st) w.n_cta_up[st] = scaled(w.n_cta_up[st], sc.other);
    }
    b->relax = fill([&](int j) { return relax_args(W[j], states[j].latents, states[j].step, 0, H[j], kRelaxNoise); },
                    [&](int j) { return scaled(relax_ctas(W[j]), sc.other); });
    {  // the entropy model: jobs with hyperlatent grids run its other form (three thread groups per
       // CTA instead of four), so the two sets of jobs get a table and a launch each; a job's bits
       // are then those of its single-image launch whatever the mix
        std::vector<ArmArgs> args(n);
        std::vector<int> o_plain, o_hyper;
        for (int j = 0; j < n; ++j) {
            args[j] = arm_args(W[j], states[j].params, H[j].lambda / (float)W[j].HW);
            ctas[j] = W[j].n_cta_arm;
        }
        for (int j : order) (W[j].g.nh > 0 ? o_hyper : o_plain).push_back(j);
        b->arm = put(tw, args, ctas, o_plain);
        b->arm_h = put(tw, args, ctas, o_hyper);
    }
    for (int m = kL - 2; m >= 1; --m)
        b->upf[m] = fill([&](int j) { return up_fwd_args(W[j], states[j].params, m); },
                         [&](int j) { return scaled(up_fwd_ctas(W[j], m), sc.other); });
    b->synf = fill([&](int j) { return syn_args(W[j], states[j].params); },
                   [&](int j) { return scaled(syn_fwd_ctas(W[j]), sc.syn); });
    b->conv = fill([&](int j) { return conv_args(W[j], states[j].params, images[j], 2.f / (3.f * (float)W[j].HW), nullptr); },
                   [&](int j) { return W[j].n_cta_conv; });
    b->synb = fill([&](int j) { return syn_args(W[j], states[j].params); }, [&](int j) { return W[j].n_cta_syn; });
    for (int st = 1; st < kL; ++st) {
        b->upa[st] = fill([&](int j) { return up_adj_args(W[j], states[j].params, st); },
                          [&](int j) { return W[j].n_cta_up[st]; });
    }
    b->ifce = fill([&](int j) { return ifce_args(W[j]); }, [&](int j) { return scaled(ifce_ctas(W[j]), sc.other); });
    b->gather = fill([&](int j) { return gather_args(W[j], kRelaxNoise, nullptr, states[j].latents, states[j].m_lat, states[j].v_lat, H[j], states[j].step, 0); },
                     [&](int j) { return scaled(gather_ctas(W[j]), sc.other); });
    b->gather_next = fill([&](int j) { return gather_args(W[j], kRelaxNoise, nullptr, states[j].latents, states[j].m_lat, states[j].v_lat, H[j], states[j].step, 0, true); },
                          [&](int j) { return scaled(gather_ctas(W[j]), sc.other); });
    b->reduce = fill([&](int j) { return reduce_args(W[j], states[j].params, states[j].m_par, states[j].v_par, nullptr, 1.f, H[j], states[j].step); },
                     [&](int) { return reduce_ctas(); });
    b->soap = fill([&](int j) { return soap_args(W[j], states[j].params, states[j].m_par, states[j].v_par,
                                                 states[j].soap, H[j], states[j].step); },
                   [&](int) { return kSoapBlocks; });
    for (int j = 0; j < n; ++j) {
        b->any_soap |= H[j].nn_opt == 1;
    }
    b->finish = fill([&](int j) {
                         // record pointer: offset of this job's first slot inside the table (fixed up below)
                         return finish_args(W[j], H[j], 1, 1, reinterpret_cast<double*>(rd_off + (size_t)j * 3 * sizeof(double)),
                                            3 * n, states[j].step, 0, 1);
                     },
                     [&](int) { return 1; });
    if (tw.host.size() > table_size) {
        delete b;
        return set_error(CC_ERR_WORKSPACE, "batch_create: table too small (%zu needed)", tw.host.size());
    }
    // place: fix up offsets into device pointers, including the record pointers inside FinishArgs
    char* base = (char*)table;
    {
        const size_t oa = reinterpret_cast<size_t>(b->finish.args);
        for (int q = 0; q < n; ++q) {
            FinishArgs fa;
            std::memcpy(&fa, tw.host.data() + oa + sizeof(FinishArgs) * q, sizeof(fa));
            fa.rd = rd_capacity > 0 ? reinterpret_cast<double*>(base + reinterpret_cast<size_t>(fa.rd)) : nullptr;
            std::memcpy(tw.host.data() + oa + sizeof(FinishArgs) * q, &fa, sizeof(fa));
        }
    }
    place(b->relax, base);
    place(b->arm, base);
    place(b->arm_h, base);
    for (int m = 1; m <= kL - 2; ++m) place(b->upf[m], base);
    place(b->synf, base);
    place(b->conv, base);
    place(b->synb, base);
    for (int st = 1; st < kL; ++st) place(b->upa[st], base);
    place(b->ifce, base);
    place(b->gather, base);
    place(b->gather_next, base);
    place(b->reduce, base);
    place(b->soap, base);
    place(b->finish, base);
    b->rd = rd_capacity > 0 ? reinterpret_cast<double*>(base + rd_off) : nullptr;
    b->table = base;
    cudaError_t e;
    if (host_staging) {
        std::memcpy(host_staging, tw.host.data(), tw.host.size());
        e = cudaMemcpyAsync(table, host_staging, tw.host.size(), cudaMemcpyHostToDevice, stream);
    } else {
        e = cudaMemcpy(table, tw.host.data(), tw.host.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        delete b;
        return set_error(CC_ERR_CUDA, "batch_create: table upload: %s", cudaGetErrorString(e));
    }
    *out = b;
    return CC_OK;
}
}  // namespace
}  // namespace cc

extern "C" {

int coolchic_batch_create(int32_t n, const cc_arch_t* archs, const cc_hparams_t* hps, const float* const* images,
                          const cc_state_t* states, void* const* workspaces, const size_t* ws_bytes,
                          const cc_schedule_t* sched, int32_t rd_capacity, void* table, size_t table_size,
                          cc_batch_t** out) {
    return batch_create_impl(n, archs, hps, images, states, workspaces, ws_bytes, sched, rd_capacity, table,
                             table_size, nullptr, nullptr, out);
}

int coolchic_batch_create_async(int32_t n, const cc_arch_t* archs, const cc_hparams_t* hps,
                                const float* const* images, const cc_state_t* states, void* const* workspaces,
                                const size_t* ws_bytes, const cc_schedule_t* sched, int32_t rd_capacity, void* table,
                                size_t table_size, void* host_staging, void* stream, cc_batch_t** out) {
    if (!host_staging) return set_error(CC_ERR_ARG, "batch_create_async: NULL host staging buffer");
    return batch_create_impl(n, archs, hps, images, states, workspaces, ws_bytes, sched, rd_capacity, table,
                             table_size, host_staging, (cudaStream_t)stream, out);
}

int coolchic_batch_step(cc_batch_t* b, int32_t n_iters, void* stream) {
    if (!b) return set_error(CC_ERR_ARG, "batch_step: NULL batch");
    if (n_iters < 0 || (b->rd_capacity > 0 && n_iters > b->rd_capacity))
        return set_error(CC_ERR_ARG, "batch_step: n_iters must lie in 0..%d (the record capacity)", b->rd_capacity);
    cudaStream_t s = (cudaStream_t)stream;
    if (b->rd) launch_mark_base_b(b->finish, s);
    for (int it = 0; it < n_iters; ++it) {
        if (it == 0) launch_relax_b(b->relax, s);  // later iterations: relaxed by the previous Adam update
        if (b->arm.njobs > 0) launch_arm_b(b->arm, PASS_FWD_BWD, false, s);
        if (b->arm_h.njobs > 0) launch_arm_b(b->arm_h, PASS_FWD_BWD, true, s);
        for (int m = kUpArmLo - 1; m >= 1; --m) launch_up_fwd_b(b->upf[m], s);  // the rest in the entropy-model launch
        launch_syn_fwd_b(b->synf, s);
        launch_conv_b(b->conv, s);
        launch_syn_bwd_b(b->synb, s);
        for (int st = 1; st < kL; ++st) launch_up_adj_b(b->upa[st], s);
        launch_ifce_b(b->ifce, s);
        launch_gather_b(it + 1 < n_iters ? b->gather_next : b->gather, s);
        launch_reduce_b(b->reduce, s);
        if (b->any_soap) launch_soap_b(b->soap, s);
        launch_finish_b(b->finish, s);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CC_ERR_CUDA, "batch_step: %s", cudaGetErrorString(e));
    return CC_OK;
}

const cc_rd_t* coolchic_batch_records(const cc_batch_t* b) { return b ? reinterpret_cast<const cc_rd_t*>(b->rd) : nullptr; }

int coolchic_batch_destroy(cc_batch_t* b) {
    delete b;
    return CC_OK;
}

}  // extern "C"
