// bfi_cli -- an integrand program speaking the line protocol of Sec. 3
// (Listings 1-2), running on the GPU through the C ABI of bfi.h.
//
// Every input line is the number of samples followed by the extent of the
// integration volume in every dimension, "n lo_1 hi_1 ... lo_d hi_d" (n may be
// written as a float, e.g. 1e7).  Every output line is the result, its
// absolute error and the dimension in which to split the volume should the
// estimate not have converged, "result abs_error split_dim".
//
// Integrands:
//   nsphere  f(x) = sqrt(max(0, 1 - |x|^2)), d taken from the line (<= 32);
//            over [-1,1]^k the result is half the volume of the unit
//            (k+1)-ball.  The split dimension is the coordinate across which f
//            is least even.
//   burgers  the weight exp(-S) of the lattice action of Eq. (Gen2), d = nx*nt
//            (a line with a single pair "lo hi" applies it to every
//            coordinate).  --output chooses the printed quantity: z (the
//            integral Z of exp(-S) over the volume), logz (ln Z and the
//            relative error of Z) or c<r> (the correlation C(r) of Eq. (C)).
//            The split dimension is the widest side, the first on ties.
//
// Line k (0-based) draws its points with Philox key (seed, k), so every line
// is an independent estimate and a rerun repeats it exactly.
//
// --adaptive is the paper's wrapper (Listing 1) instead: no standard input;
// the volume [min-extent, max-extent]^dimensions is subdivided until every
// subvolume passes the convergence test of Sec. 3 (--samples n, --factor,
// --rel-tol, --abs-tol, --small, --max-depth, --max-leaves) and one line
// "result abs_error" is written.
#include "bfi.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace {

void usage(const char *prog) {
    std::fprintf(stderr,
                 "usage: %s [--integrand nsphere|burgers] [--seed S] [--device K]\n"
                 "          [--lattice NXxNT] [--nu X] [--D X] [--a X] [--tau X] [--nonlinear X] [--mass2 X]\n"
                 "          [--precision fp64|fp32] [--output z|logz|c<r>]\n"
                 "          [--adaptive 1 --dimensions K --min-extent A --max-extent B --samples N\n"
                 "           --factor F --rel-tol X --abs-tol X --small X --max-depth K --max-leaves K]\n"
                 "reads lines 'n lo_1 hi_1 ... lo_d hi_d' from standard input and writes\n"
                 "'result abs_error split_dim' for each; with --adaptive 1, integrates\n"
                 "[A, B]^K adaptively and writes 'result abs_error'\n",
                 prog);
}

struct Options {
    std::string integrand = "nsphere";
    uint32_t seed = 1;
    int device = 0;
    bfi_lattice lat{10, 2, 1.0, 1.0, 1.0, 1.0, 1.0, 0.0};
    bfi_precision precision = BFI_FP64;
    std::string output = "z";
    bool adaptive = false;
    int dims = 0;
    double min_extent = -1.0, max_extent = 1.0, samples = 1e5;
    bfi_convergence conv{2.0, 1e-2, 0.0, 0.0, 12, 1 << 16};
};

bool parse_double(const char *s, double *out) {
    char *end = nullptr;
    *out = std::strtod(s, &end);
    return end != s && *end == '\0';
}

int parse_options(int argc, char **argv, Options *o) {
    for (int i = 1; i < argc; ++i) {
        const std::string k = argv[i];
        if (k == "-h" || k == "--help") {
            usage(argv[0]);
            std::exit(0);
        }
        if (i + 1 >= argc) {
            std::fprintf(stderr, "option %s needs a value\n", k.c_str());
            return 2;
        }
        const char *v = argv[++i];
        double x = 0.0;
        if (k == "--integrand") {
            o->integrand = v;
            if (o->integrand != "nsphere" && o->integrand != "burgers") {
                std::fprintf(stderr, "unknown integrand %s\n", v);
                return 2;
            }
        } else if (k == "--seed" && parse_double(v, &x) && x >= 0 && x < 4294967296.0) {
            o->seed = static_cast<uint32_t>(x);
        } else if (k == "--device" && parse_double(v, &x) && x >= 0) {
            o->device = static_cast<int>(x);
        } else if (k == "--lattice") {
            int nx = 0, nt = 0;
            if (std::sscanf(v, "%dx%d", &nx, &nt) != 2) {
                std::fprintf(stderr, "--lattice wants NXxNT, e.g. 10x2\n");
                return 2;
            }
            o->lat.nx = nx;
            o->lat.nt = nt;
        } else if (k == "--nu" && parse_double(v, &x)) {
            o->lat.nu = x;
        } else if (k == "--D" && parse_double(v, &x)) {
            o->lat.D = x;
        } else if (k == "--a" && parse_double(v, &x)) {
            o->lat.a = x;
        } else if (k == "--tau" && parse_double(v, &x)) {
            o->lat.tau = x;
        } else if (k == "--nonlinear" && parse_double(v, &x)) {
            o->lat.nonlinear = x;
        } else if (k == "--mass2" && parse_double(v, &x)) {
            o->lat.mass2 = x;
        } else if (k == "--precision" && (!std::strcmp(v, "fp64") || !std::strcmp(v, "fp32"))) {
            o->precision = std::strcmp(v, "fp64") ? BFI_FP32 : BFI_FP64;
        } else if (k == "--output") {
            o->output = v;
        } else if (k == "--adaptive" && parse_double(v, &x)) {
            o->adaptive = x != 0.0;
        } else if (k == "--dimensions" && parse_double(v, &x) && x >= 1 && x <= 32) {
            o->dims = static_cast<int>(x);
        } else if (k == "--min-extent" && parse_double(v, &x)) {
            o->min_extent = x;
        } else if (k == "--max-extent" && parse_double(v, &x)) {
            o->max_extent = x;
        } else if (k == "--samples" && parse_double(v, &x)) {
            o->samples = x;
        } else if (k == "--factor" && parse_double(v, &x)) {
            o->conv.factor = x;
        } else if (k == "--rel-tol" && parse_double(v, &x)) {
            o->conv.rel_tol = x;
        } else if (k == "--abs-tol" && parse_double(v, &x)) {
            o->conv.abs_tol = x;
        } else if (k == "--small" && parse_double(v, &x)) {
            o->conv.small = x;
        } else if (k == "--max-depth" && parse_double(v, &x) && x >= 0 && x <= 30) {
            o->conv.max_depth = static_cast<int32_t>(x);
        } else if (k == "--max-leaves" && parse_double(v, &x) && x >= 1) {
            o->conv.max_leaves = static_cast<int64_t>(x);
        } else {
            std::fprintf(stderr, "bad option or value: %s %s\n", k.c_str(), v);
            usage(argv[0]);
            return 2;
        }
    }
    if (o->integrand == "burgers") {
        const std::string &out = o->output;
        bool ok = out == "z" || out == "logz";
        if (!ok && out.size() > 1 && out[0] == 'c') {
            char *end = nullptr;
            const long r = std::strtol(out.c_str() + 1, &end, 10);
            ok = *end == '\0' && r >= 0 && r <= o->lat.nx / 2;
        }
        if (!ok) {
            std::fprintf(stderr, "--output wants z, logz or c<r> with 0 <= r <= nx/2\n");
            return 2;
        }
    }
    return 0;
}

// Splits a line into numbers; false on anything that is not a number.
bool numbers(const std::string &line, std::vector<double> *out) {
    out->clear();
    const char *p = line.c_str();
    while (*p) {
        while (*p == ' ' || *p == '\t' || *p == '\r' || *p == '\n') ++p;
        if (!*p) break;
        char *end = nullptr;
        const double v = std::strtod(p, &end);
        if (end == p) return false;
        out->push_back(v);
        p = end;
    }
    return true;
}

int fail(const char *what) {
    std::fprintf(stderr, "%s: %s\n", what, bfi_last_error());
    return 3;
}

// The wrapper of Listing 1: adaptive subdivision of one cube.
int run_adaptive(const Options &o) {
    const bool burgers = o.integrand == "burgers";
    const int d = burgers ? o.lat.nx * o.lat.nt : o.dims;
    if (d < 1 || !(o.max_extent > o.min_extent) || !(o.samples >= 2.0) || o.samples != std::floor(o.samples) ||
        o.samples >= 281474976710656.0) {
        std::fprintf(stderr, "--adaptive needs --dimensions (nsphere), min-extent < max-extent and an integer "
                             "--samples >= 2\n");
        return 2;
    }
    const uint64_t n = static_cast<uint64_t>(o.samples);
    std::vector<double> lo(d, o.min_extent), hi(d, o.max_extent);
    double result = 0.0, err = 0.0;
    if (!burgers) {
        const bfi_status st = bfi_adaptive_nsphere(d, lo.data(), hi.data(), n, o.seed, 0u, &o.conv, &result, &err,
                                                   nullptr, o.device);
        if (st != BFI_OK) return st == BFI_E_INVALID ? (fail("bfi_adaptive_nsphere"), 2) : fail("bfi_adaptive_nsphere");
    } else {
        bfi_ctx *ctx = nullptr;
        if (bfi_ctx_create(&ctx, o.device) != BFI_OK) return fail("bfi_ctx_create");
        std::vector<double> totals(bfi_totals_len(o.lat.nx));
        const bfi_status st = bfi_adaptive_integrate(ctx, &o.lat, lo.data(), hi.data(), n, o.seed, 0u, o.precision,
                                                     &o.conv, totals.data(), nullptr, 0, nullptr, nullptr, nullptr);
        bfi_ctx_destroy(ctx);
        if (st != BFI_OK) return st == BFI_E_INVALID ? (fail("bfi_adaptive_integrate"), 2) : fail("bfi_adaptive_integrate");
        const int R = bfi_num_r(o.lat.nx);
        if (o.output == "z") {
            result = std::exp(totals[0]);
            err = result * totals[1];
        } else if (o.output == "logz") {
            result = totals[0];
            err = totals[1];
        } else {
            const int r = std::atoi(o.output.c_str() + 1);
            result = totals[4 + r];
            err = totals[4 + R + r];
        }
    }
    std::printf("%.15g %.15g\n", result, err);
    return 0;
}

}  // namespace

int main(int argc, char **argv) {
    Options o;
    if (const int rc = parse_options(argc, argv, &o)) return rc;
    if (o.adaptive) return run_adaptive(o);
    const bool burgers = o.integrand == "burgers";
    const int d = o.lat.nx * o.lat.nt;
    bfi_ctx *ctx = nullptr;
    std::vector<double> slots, totals;
    if (burgers) {
        if (bfi_ctx_create(&ctx, o.device) != BFI_OK) return fail("bfi_ctx_create");
        slots.resize(bfi_slot_len(o.lat.nx));
        totals.resize(bfi_totals_len(o.lat.nx));
    }
    std::string line;
    std::vector<double> v, lo, hi;
    char buf[1 << 14];
    uint32_t job = 0;
    int rc = 0;
    while (std::fgets(buf, sizeof buf, stdin)) {
        line.assign(buf);
        while (line.size() == sizeof buf - 1 && line.back() != '\n' && std::fgets(buf, sizeof buf, stdin)) line += buf;
        if (!numbers(line, &v)) {
            std::fprintf(stderr, "line %u: not a list of numbers\n", job);
            rc = 2;
            break;
        }
        if (v.empty()) continue;
        const double nd = v[0];
        if (!(nd >= 2.0) || nd != std::floor(nd) || nd >= 281474976710656.0) {
            std::fprintf(stderr, "line %u: the sample count must be an integer in [2, 2^48)\n", job);
            rc = 2;
            break;
        }
        const uint64_t n = static_cast<uint64_t>(nd);
        const size_t pairs = (v.size() - 1) / 2;
        if (v.size() % 2 != 1 || pairs < 1 || (burgers && pairs != 1 && pairs != static_cast<size_t>(d))) {
            std::fprintf(stderr, "line %u: expected n followed by %s lo/hi pairs\n", job,
                         burgers ? (std::to_string(d) + " (or 1)").c_str() : "d");
            rc = 2;
            break;
        }
        const size_t dims = burgers ? static_cast<size_t>(d) : pairs;
        lo.assign(dims, 0.0);
        hi.assign(dims, 0.0);
        bool ordered = true;
        for (size_t j = 0; j < dims; ++j) {
            const size_t q = pairs == 1 ? 0 : j;
            lo[j] = v[1 + 2 * q];
            hi[j] = v[2 + 2 * q];
            ordered = ordered && hi[j] > lo[j];
        }
        if (!ordered) {
            std::fprintf(stderr, "line %u: need lo < hi in every dimension\n", job);
            rc = 2;
            break;
        }
        double result = 0.0, err = 0.0;
        int32_t split = 0;
        if (!burgers) {
            if (bfi_nsphere(static_cast<int32_t>(dims), lo.data(), hi.data(), n, o.seed, job, 0u, &result, &err,
                            &split, o.device) != BFI_OK) {
                rc = fail("bfi_nsphere");
                break;
            }
        } else {
            if (bfi_integrate(ctx, &o.lat, 1, lo.data(), hi.data(), &n, nullptr, o.seed, job, o.precision,
                              slots.data(), totals.data()) != BFI_OK) {
                rc = fail("bfi_integrate");
                break;
            }
            const int R = bfi_num_r(o.lat.nx);
            if (o.output == "z") {
                result = std::exp(totals[0]);
                err = result * totals[1];
            } else if (o.output == "logz") {
                result = totals[0];
                err = totals[1];
            } else {
                const int r = std::atoi(o.output.c_str() + 1);
                result = totals[4 + r];
                err = totals[4 + R + r];
            }
            double widest = -1.0;
            for (size_t j = 0; j < dims; ++j)
                if (hi[j] - lo[j] > widest) {
                    widest = hi[j] - lo[j];
                    split = static_cast<int32_t>(j);
                }
        }
        std::printf("%.15e %.15e %d\n", result, err, split);
        std::fflush(stdout);
        ++job;
    }
    if (ctx) bfi_ctx_destroy(ctx);
    return rc;
}
