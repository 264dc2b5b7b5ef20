// adaptive.cu -- adaptive subdivision with the convergence test of Sec. 3
// (host code).  Each round evaluates every open subvolume twice, with n and
// factor * n samples, in a single GPU launch (the N-sphere batch or one
// lattice plan over all 2k evaluations), then keeps the converged ones and
// halves the rest.  The paper's wrapper ran one integrand process per
// subvolume and evaluation; here a round is one launch.
#include "bfi.h"
#include "bfi_host.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

constexpr int kMaxDepth = 30;  // heap numbers of depth <= 30 stay below 2^31, sub_ids below 2^32

struct Node {
    uint32_t heap;
    int32_t depth;
};

// The open subvolumes of one round, in order.
struct Front {
    int d = 0;
    std::vector<double> lo, hi;  // [k][d]
    std::vector<Node> nodes;
    size_t size() const { return nodes.size(); }
    void push(const double *l, const double *h, Node nd) {
        lo.insert(lo.end(), l, l + d);
        hi.insert(hi.end(), h, h + d);
        nodes.push_back(nd);
    }
    void clear() {
        lo.clear();
        hi.clear();
        nodes.clear();
    }
};

bfi_status check_convergence(const bfi_convergence *c, uint64_t n, uint64_t *n2) {
    if (!c) return bfi::set_error(BFI_E_INVALID, "conv is NULL");
    if (!(c->factor >= 1.0) || !(c->factor <= 1e6))
        return bfi::set_error(BFI_E_INVALID, "factor must lie in [1, 1e6]");
    if (c->max_depth < 0 || c->max_depth > kMaxDepth) return bfi::set_error(BFI_E_INVALID, "max_depth must lie in [0, 30]");
    if (c->max_leaves < 1) return bfi::set_error(BFI_E_INVALID, "max_leaves must be >= 1");
    if (std::isnan(c->rel_tol) || std::isnan(c->abs_tol) || std::isnan(c->small))
        return bfi::set_error(BFI_E_INVALID, "a threshold is NaN");
    if (n < 2 || n >= (uint64_t(1) << 48)) return bfi::set_error(BFI_E_INVALID, "n must lie in [2, 2^48)");
    const double m = std::ceil(c->factor * static_cast<double>(n));
    if (!(m < 281474976710656.0)) return bfi::set_error(BFI_E_INVALID, "factor * n must be < 2^48");
    *n2 = static_cast<uint64_t>(m);
    return BFI_OK;
}

// The three criteria of Sec. 3 on two results; (1) is the ratio test of
// Sec. 4 (results within a factor 1 + rel_tol of each other).
bool converged_linear(double r1, double r2, const bfi_convergence &c) {
    const double diff = std::fabs(r1 - r2), big = std::fmax(std::fabs(r1), std::fabs(r2)),
                 little = std::fmin(std::fabs(r1), std::fabs(r2));
    return (c.rel_tol > 0.0 && diff <= c.rel_tol * little) || (c.abs_tol > 0.0 && diff <= c.abs_tol) ||
           (c.small > 0.0 && big <= c.small);
}

// The same criteria for positive results given by their logarithms:
// |Z1 - Z2| / min(Z1, Z2) = exp(|ln Z1 - ln Z2|) - 1.
bool converged_log(double l1, double l2, const bfi_convergence &c) {
    const double top = std::fmax(l1, l2), rel = std::expm1(std::fabs(l1 - l2));
    const double low = std::fmin(l1, l2);
    return (c.rel_tol > 0.0 && rel <= c.rel_tol) || (c.abs_tol > 0.0 && std::exp(low) * rel <= c.abs_tol) ||
           (c.small > 0.0 && top <= std::log(c.small));
}

enum class Fate { kConverged, kDepth, kBudget, kSplit };

// Decisions of one round in order: a subvolume that has not converged is
// halved while the next round has room for both halves.
void decide(const Front &f, const std::vector<bool> &conv, const bfi_convergence &c, std::vector<Fate> *fate) {
    fate->assign(f.size(), Fate::kConverged);
    int64_t next = 0;
    for (size_t i = 0; i < f.size(); ++i) {
        if (conv[i]) continue;
        if (f.nodes[i].depth >= c.max_depth) {
            (*fate)[i] = Fate::kDepth;
        } else if (next + 2 <= c.max_leaves) {
            (*fate)[i] = Fate::kSplit;
            next += 2;
        } else {
            (*fate)[i] = Fate::kBudget;
        }
    }
}

void split(const Front &f, size_t i, int dim, Front *next) {
    const int d = f.d;
    std::vector<double> l(f.lo.begin() + i * d, f.lo.begin() + (i + 1) * d);
    std::vector<double> h(f.hi.begin() + i * d, f.hi.begin() + (i + 1) * d);
    const double mid = 0.5 * (l[dim] + h[dim]);
    const Node nd = f.nodes[i];
    std::vector<double> h_low = h, l_up = l;
    h_low[dim] = mid;
    l_up[dim] = mid;
    next->push(l.data(), h_low.data(), Node{2 * nd.heap, nd.depth + 1});
    next->push(l_up.data(), h.data(), Node{2 * nd.heap + 1, nd.depth + 1});
}

void count(Fate fate, bfi_adaptive_stats *st) {
    if (fate == Fate::kConverged) ++st->converged;
    if (fate == Fate::kDepth) ++st->kept_depth;
    if (fate == Fate::kBudget) ++st->kept_budget;
    if (fate != Fate::kSplit) ++st->leaves;
}

// Both evaluations of every subvolume of a round: boxes [A_0..A_{k-1},
// B_0..B_{k-1}] with n and n2 samples and sub_ids 2h and 2h + 1.
void round_inputs(const Front &f, uint64_t n, uint64_t n2, std::vector<double> *lo, std::vector<double> *hi,
                  std::vector<uint64_t> *smp, std::vector<uint32_t> *sid) {
    const size_t k = f.size();
    lo->assign(f.lo.begin(), f.lo.end());
    lo->insert(lo->end(), f.lo.begin(), f.lo.end());
    hi->assign(f.hi.begin(), f.hi.end());
    hi->insert(hi->end(), f.hi.begin(), f.hi.end());
    smp->assign(2 * k, n);
    sid->resize(2 * k);
    for (size_t i = 0; i < k; ++i) {
        (*smp)[k + i] = n2;
        (*sid)[i] = 2u * f.nodes[i].heap;
        (*sid)[k + i] = 2u * f.nodes[i].heap + 1u;
    }
}

bfi_status check_box(int d, const double *lo, const double *hi) {
    if (!lo || !hi) return bfi::set_error(BFI_E_INVALID, "lo or hi is NULL");
    for (int j = 0; j < d; ++j)
        if (!(hi[j] > lo[j]) || !std::isfinite(lo[j]) || !std::isfinite(hi[j]))
            return bfi::set_error(BFI_E_INVALID, "need finite lo < hi in every coordinate");
    return BFI_OK;
}

}  // namespace

extern "C" {

bfi_status bfi_adaptive_nsphere(int32_t dims, const double *lo, const double *hi, uint64_t n, uint32_t seed,
                                uint32_t job_id, const bfi_convergence *conv, double *result, double *abs_err,
                                bfi_adaptive_stats *stats, int device) {
    uint64_t n2 = 0;
    bfi_status st = check_convergence(conv, n, &n2);
    if (st != BFI_OK) return st;
    if (dims < 1 || dims > 32) return bfi::set_error(BFI_E_INVALID, "need 1 <= dims <= 32");
    if ((st = check_box(dims, lo, hi)) != BFI_OK) return st;
    if (!result || !abs_err) return bfi::set_error(BFI_E_INVALID, "result or abs_err is NULL");
    bfi_adaptive_stats s{};
    Front front, next;
    front.d = next.d = dims;
    front.push(lo, hi, Node{1u, 0});
    double sum = 0.0, var = 0.0;
    std::vector<double> blo, bhi, sums;
    std::vector<uint64_t> smp;
    std::vector<uint32_t> sid;
    std::vector<bool> conv_i;
    std::vector<Fate> fate;
    std::vector<double> r2(0), e2(0);
    std::vector<int32_t> sd(0);
    while (front.size() > 0) {
        const size_t k = front.size();
        ++s.rounds;
        s.evaluated += static_cast<int64_t>(k);
        s.samples += static_cast<uint64_t>(k) * (n + n2);
        round_inputs(front, n, n2, &blo, &bhi, &smp, &sid);
        sums.resize(2 * k * (2 + dims));
        st = bfi::nsphere_batch(dims, static_cast<int64_t>(2 * k), blo.data(), bhi.data(), smp.data(), sid.data(),
                                seed, job_id, device, sums.data());
        if (st != BFI_OK) return st;
        conv_i.assign(k, false);
        r2.resize(k);
        e2.resize(k);
        sd.resize(k);
        for (size_t i = 0; i < k; ++i) {
            double r1 = 0.0, e1 = 0.0;
            const double *l = front.lo.data() + i * dims, *h = front.hi.data() + i * dims;
            bfi::nsphere_finish(dims, l, h, n, sums.data() + i * (2 + dims), &r1, &e1, nullptr);
            bfi::nsphere_finish(dims, l, h, n2, sums.data() + (k + i) * (2 + dims), &r2[i], &e2[i], &sd[i]);
            conv_i[i] = converged_linear(r1, r2[i], *conv);
        }
        decide(front, conv_i, *conv, &fate);
        next.clear();
        for (size_t i = 0; i < k; ++i) {
            count(fate[i], &s);
            if (fate[i] == Fate::kSplit) {
                split(front, i, sd[i], &next);
            } else {
                sum += r2[i];
                var += e2[i] * e2[i];
            }
        }
        std::swap(front, next);
    }
    *result = sum;
    *abs_err = std::sqrt(var);
    if (stats) *stats = s;
    return BFI_OK;
}

bfi_status bfi_adaptive_integrate(bfi_ctx *ctx, const bfi_lattice *lattice, const double *lo, const double *hi,
                                  uint64_t n, uint32_t seed, uint32_t job_id, bfi_precision precision,
                                  const bfi_convergence *conv, double *totals, bfi_adaptive_stats *stats,
                                  int64_t leaf_capacity, double *leaf_lo, double *leaf_hi, double *leaf_slots) {
    if (!ctx) return bfi::set_error(BFI_E_INVALID, "ctx is NULL");
    bfi_status st = bfi::validate_lattice(lattice);
    if (st != BFI_OK) return st;
    uint64_t n2 = 0;
    if ((st = check_convergence(conv, n, &n2)) != BFI_OK) return st;
    const int d = lattice->nx * lattice->nt;
    if ((st = check_box(d, lo, hi)) != BFI_OK) return st;
    if (!totals) return bfi::set_error(BFI_E_INVALID, "totals is NULL");
    if (leaf_capacity < 0) return bfi::set_error(BFI_E_INVALID, "leaf_capacity is negative");
    const int L = bfi_slot_len(lattice->nx);
    bfi_adaptive_stats s{};
    Front front, next;
    front.d = next.d = d;
    front.push(lo, hi, Node{1u, 0});
    std::vector<double> blo, bhi, slots, kept, tmp_totals(bfi_totals_len(lattice->nx));
    std::vector<uint64_t> smp;
    std::vector<uint32_t> sid;
    std::vector<bool> conv_i;
    std::vector<Fate> fate;
    std::vector<int> widest;
    int64_t written = 0;
    while (front.size() > 0) {
        const size_t k = front.size();
        ++s.rounds;
        s.evaluated += static_cast<int64_t>(k);
        s.samples += static_cast<uint64_t>(k) * (n + n2);
        round_inputs(front, n, n2, &blo, &bhi, &smp, &sid);
        slots.resize(2 * k * L);
        st = bfi_integrate(ctx, lattice, static_cast<int64_t>(2 * k), blo.data(), bhi.data(), smp.data(), sid.data(),
                           seed, job_id, precision, slots.data(), tmp_totals.data());
        if (st != BFI_OK) return st;
        conv_i.assign(k, false);
        widest.assign(k, 0);
        for (size_t i = 0; i < k; ++i) {
            // ln Z_s = ln V_s - ln n_s - m_s + ln sum w
            const double *a = slots.data() + i * L, *b = slots.data() + (k + i) * L;
            const double l1 = a[2] - std::log(a[0]) - a[1] + std::log(a[3]);
            const double l2 = b[2] - std::log(b[0]) - b[1] + std::log(b[3]);
            conv_i[i] = converged_log(l1, l2, *conv);
            const double *bl = front.lo.data() + i * d, *bh = front.hi.data() + i * d;
            double w_best = -1.0;
            for (int j = 0; j < d; ++j)
                if (bh[j] - bl[j] > w_best) {
                    w_best = bh[j] - bl[j];
                    widest[i] = j;
                }
        }
        decide(front, conv_i, *conv, &fate);
        next.clear();
        for (size_t i = 0; i < k; ++i) {
            count(fate[i], &s);
            if (fate[i] == Fate::kSplit) {
                split(front, i, widest[i], &next);
                continue;
            }
            const double *b = slots.data() + (k + i) * L;
            kept.insert(kept.end(), b, b + L);
            if (written < leaf_capacity) {
                if (leaf_lo) std::memcpy(leaf_lo + written * d, front.lo.data() + i * d, sizeof(double) * d);
                if (leaf_hi) std::memcpy(leaf_hi + written * d, front.hi.data() + i * d, sizeof(double) * d);
                if (leaf_slots) std::memcpy(leaf_slots + written * L, b, sizeof(double) * L);
                ++written;
            }
        }
        std::swap(front, next);
    }
    st = bfi_merge_host(lattice->nx, static_cast<int64_t>(kept.size() / L), kept.data(), totals);
    if (st != BFI_OK) return st;
    if (stats) *stats = s;
    return BFI_OK;
}

}  // extern "C"
