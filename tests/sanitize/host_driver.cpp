// Host-code driver for the address and undefined-behaviour sanitizers: the CSR builder,
// the recursive bisection (Algorithm 1), the relabelling and the graph-file reader and
// writer, on random multigraphs and on malformed files.  Built and run by
// tests/test_host_sanitize.py with -fsanitize=address,undefined; exits non-zero on any
// broken invariant, and the sanitizers abort on any memory or UB error.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "rn_internal.h"

static int failures = 0;
#define CHECK(c)                                                                  \
    do {                                                                          \
        if (!(c)) {                                                               \
            std::fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #c); \
            failures++;                                                           \
        }                                                                         \
    } while (0)

static void graphs(uint32_t seed) {
    std::mt19937 rng(seed);
    const uint32_t n = 1 + rng() % 1200;
    const uint64_t m = rng() % (4 * uint64_t(n) + 1);
    std::vector<uint32_t> src(m), dst(m), w(m);
    for (uint64_t i = 0; i < m; i++) {
        src[i] = rng() % n;
        dst[i] = (rng() % 5 == 0) ? src[i] : rng() % n;  // self-loops and parallel arcs too
        w[i] = 1 + rng() % 1000;
    }
    for (bool undirected : {true, false}) {
        rn::HostGraph g = rn::build_csr(n, m, src.data(), dst.data(), w.data(), undirected);
        CHECK(g.n == n && g.row_ptr.size() == size_t(n) + 1 && g.row_ptr[n] == g.arcs());
        for (uint32_t x = 0; x < n; x++)
            for (uint32_t e = g.row_ptr[x]; e < g.row_ptr[x + 1]; e++) {
                CHECK(g.col[e] < n && g.col[e] != x && g.w[e] >= 1);
                if (e > g.row_ptr[x]) CHECK(g.col[e - 1] < g.col[e]);  // one arc per head
            }
        for (uint32_t leaf : {1u, 7u, 512u}) {
            for (float alpha : {0.0f, 0.5f, 1.0f}) {
                std::vector<uint32_t> order = rn::bisection_order(g, leaf, alpha, undirected);
                CHECK(order.size() == n);
                std::vector<char> seen(n, 0);
                for (uint32_t v : order) {
                    CHECK(v < n && !seen[v]);
                    if (v < n) seen[v] = 1;
                }
                rn::HostGraph r = rn::relabel(g, order);
                CHECK(r.arcs() == g.arcs() && r.n == n);
            }
        }
    }
}

static void files(uint32_t seed, const std::string &dir) {
    std::mt19937 rng(seed);
    const uint32_t n = 1 + rng() % 500;
    const uint64_t m = rng() % 2000;
    std::vector<uint32_t> src(m), dst(m), w(m);
    for (uint64_t i = 0; i < m; i++) {
        src[i] = rng() % n;
        dst[i] = rng() % n;
        w[i] = 1 + rng() % 100;
    }
    const std::string path = dir + "/g" + std::to_string(seed) + ".rng";
    rn::write_edge_file(path.c_str(), n, m, src.data(), dst.data(), w.data(), RN_UNDIRECTED);
    rn::EdgeFile f;
    rn::read_edge_file(path.c_str(), &f);
    CHECK(f.n == n && f.flags == RN_UNDIRECTED && f.src == src && f.dst == dst && f.w == w);
    // every truncation of the file is rejected
    std::FILE *in = std::fopen(path.c_str(), "rb");
    std::vector<char> bytes;
    for (int c; (c = std::fgetc(in)) != EOF;) bytes.push_back(char(c));
    std::fclose(in);
    for (size_t cut : {size_t(0), size_t(3), size_t(12), bytes.size() / 2, bytes.size() - 1}) {
        if (cut >= bytes.size()) continue;
        const std::string t = dir + "/cut.rng";
        std::FILE *o = std::fopen(t.c_str(), "wb");
        std::fwrite(bytes.data(), 1, cut, o);
        std::fclose(o);
        bool threw = false;
        try {
            rn::read_edge_file(t.c_str(), &f);
        } catch (const rn::Error &) {
            threw = true;
        }
        CHECK(threw);
    }
    // DIMACS text with junk
    const std::string gr = dir + "/g.gr";
    for (const char *text : {"p sp 3 2\na 1 2 5\na 2 3 7\n", "p sp 3 1\na 1 9 5\n", "a 1 2 3\n", "p sp 2 1\nzz\n",
                             "c only comments\n", "p sp 2 1\na 1 2 99999999999\n"}) {
        std::FILE *o = std::fopen(gr.c_str(), "w");
        std::fputs(text, o);
        std::fclose(o);
        try {
            rn::read_edge_file(gr.c_str(), &f);
            CHECK(f.n == 3 && f.src.size() == 2);  // only the first text is valid
        } catch (const rn::Error &) {
        }
    }
}

int main(int argc, char **argv) {
    const std::string dir = argc > 1 ? argv[1] : ".";
    for (uint32_t s = 0; s < 16; s++) graphs(s);
    for (uint32_t s = 0; s < 20; s++) files(s, dir);
    std::printf("host driver: %d failures\n", failures);
    return failures ? 1 : 0;
}
