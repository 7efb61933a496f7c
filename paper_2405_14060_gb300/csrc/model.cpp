// Model input: UAI text parsing and validation of array input (host).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>

#include "model.h"

namespace tn {

std::string validate_model(const ModelData &m) {
    if (m.nvars < 0) return "negative variable count";
    if ((int)m.card.size() != m.nvars) return "card has the wrong length";
    for (int v = 0; v < m.nvars; ++v)
        if (m.card[v] < 1) return "domain size < 1 for variable " + std::to_string(v);
    if ((int)m.scope.size() != m.nfactors) return "scope count mismatch";
    int64_t tot = 0;
    for (int f = 0; f < m.nfactors; ++f) {
        const auto &s = m.scope[f];
        int64_t sz = 1;
        for (size_t i = 0; i < s.size(); ++i) {
            int v = s[i];
            if (v < 0 || v >= m.nvars)
                return "factor " + std::to_string(f) + " has a variable out of range";
            for (size_t j = 0; j < i; ++j)
                if (s[j] == v) return "factor " + std::to_string(f) + " repeats a variable";
            sz *= m.card[v];
            if (sz > (int64_t)1 << 40) return "factor table too large";
        }
        if (m.toff[f] != tot) return "table offsets inconsistent";
        tot += sz;
    }
    if ((int64_t)m.tables.size() != tot) return "table length mismatch";
    for (int64_t i = 0; i < tot; ++i) {
        double x = m.tables[i];
        if (!(x >= 0.0) || !std::isfinite(x))
            return "factor table entry negative or not finite";
    }
    return "";
}

std::string model_from_arrays(int nvars, const int *card, int nfactors, const int *scope_off,
                              const int *scope_vars, const double *tables, ModelData &m) {
    if (nvars < 0 || nfactors < 0) return "negative size";
    if ((nvars && !card) || (nfactors && (!scope_off || !tables))) return "NULL array";
    m.nvars = nvars;
    m.card.assign(card, card + nvars);
    m.nfactors = nfactors;
    m.scope.clear();
    m.toff.clear();
    int64_t tot = 0;
    for (int f = 0; f < nfactors; ++f) {
        int a = scope_off[f], b = scope_off[f + 1];
        if (b < a) return "scope offsets decrease";
        std::vector<int> s(scope_vars + a, scope_vars + b);
        for (int v : s)
            if (v < 0 || v >= nvars) return "scope variable out of range";
        int64_t sz = 1;
        for (int v : s) sz *= card[v];
        m.scope.push_back(s);
        m.toff.push_back(tot);
        tot += sz;
    }
    m.tables.assign(tables, tables + tot);
    return validate_model(m);
}

std::string model_from_uai(const char *path, ModelData &m, bool &parse_error) {
    parse_error = false;
    std::ifstream in(path);
    if (!in) return std::string("cannot open ") + path;
    std::stringstream ss;
    ss << in.rdbuf();
    std::string kind;
    ss >> kind;
    if (kind != "MARKOV" && kind != "BAYES") {
        parse_error = true;
        return "expected MARKOV or BAYES";
    }
    int n = -1;
    if (!(ss >> n) || n < 0) { parse_error = true; return "bad variable count"; }
    std::vector<int> card(n);
    for (int v = 0; v < n; ++v)
        if (!(ss >> card[v])) { parse_error = true; return "bad domain sizes"; }
    int nf = -1;
    if (!(ss >> nf) || nf < 0) { parse_error = true; return "bad factor count"; }
    std::vector<int> off(nf + 1, 0), sv;
    for (int f = 0; f < nf; ++f) {
        int k;
        if (!(ss >> k) || k < 0) { parse_error = true; return "bad scope size"; }
        for (int i = 0; i < k; ++i) {
            int v;
            if (!(ss >> v)) { parse_error = true; return "bad scope"; }
            sv.push_back(v);
        }
        off[f + 1] = off[f] + k;
    }
    std::vector<double> tab;
    for (int f = 0; f < nf; ++f) {
        int64_t sz;
        if (!(ss >> sz) || sz < 0) { parse_error = true; return "bad table size"; }
        int64_t expect = 1;
        for (int i = off[f]; i < off[f + 1]; ++i) {
            int v = sv[i];
            if (v < 0 || v >= n) { parse_error = true; return "scope variable out of range"; }
            expect *= card[v];
        }
        if (sz != expect) { parse_error = true; return "table size does not match scope"; }
        for (int64_t i = 0; i < sz; ++i) {
            double x;
            if (!(ss >> x)) { parse_error = true; return "truncated table"; }
            tab.push_back(x);
        }
    }
    return model_from_arrays(n, card.data(), nf, off.data(), sv.data(), tab.data(), m);
}

static bool read_ints(const char *path, std::vector<long long> &t, std::string &err) {
    std::ifstream in(path);
    if (!in) {
        err = std::string("cannot open ") + path;
        return false;
    }
    std::string tok;
    while (in >> tok) {
        char *end = nullptr;
        long long v = std::strtoll(tok.c_str(), &end, 10);
        if (!end || *end) {
            err = "not an integer: " + tok;
            return false;
        }
        t.push_back(v);
    }
    return true;
}

// One block "<nobs> v1 x1 ..." starting at t[p]; false if it does not fit.
static bool evidence_block(const std::vector<long long> &t, size_t &p, size_t end) {
    if (p >= end || t[p] < 0) return false;
    long long k = t[p];
    if ((long long)(end - p - 1) < 2 * k) return false;
    p += 1 + 2 * (size_t)k;
    return true;
}

std::string evidence_from_uai(const char *path, const ModelData &m,
                              std::vector<std::vector<int32_t>> &sets, bool &parse_error) {
    parse_error = false;
    sets.clear();
    std::vector<long long> t;
    std::string err;
    if (!read_ints(path, t, err)) {
        parse_error = err.rfind("cannot open", 0) != 0;
        return err;
    }
    if (t.empty()) {
        parse_error = true;
        return "empty evidence file";
    }
    // several sets when "<nsets>" and exactly that many blocks fill the file
    std::vector<std::pair<size_t, size_t>> blocks;   // (start, end) of each block
    bool multi = false;
    if (t[0] >= 0) {
        size_t p = 1;
        std::vector<std::pair<size_t, size_t>> b;
        long long n = t[0];
        bool ok = true;
        for (long long i = 0; i < n && ok; ++i) {
            size_t s0 = p;
            ok = evidence_block(t, p, t.size());
            if (ok) b.push_back({s0, p});
        }
        if (ok && p == t.size() && !(n == 0 && t.size() == 1)) {
            multi = true;
            blocks = b;
        }
    }
    if (!multi) {
        size_t p = 0;
        if (!evidence_block(t, p, t.size()) || p != t.size()) {
            parse_error = true;
            return "evidence file is neither one block \"<nobs> var value ...\" nor a "
                   "count of such blocks followed by them";
        }
        blocks.push_back({0, p});
    }
    for (auto &b : blocks) {
        std::vector<int32_t> row(m.nvars, -1);
        long long k = t[b.first];
        for (long long i = 0; i < k; ++i) {
            long long v = t[b.first + 1 + 2 * i], x = t[b.first + 2 + 2 * i];
            if (v < 0 || v >= m.nvars) {
                parse_error = true;
                return "evidence variable out of range: " + std::to_string(v);
            }
            if (x < 0 || x >= m.card[v]) {
                parse_error = true;
                return "evidence value out of range for variable " + std::to_string(v);
            }
            if (row[v] >= 0) {
                parse_error = true;
                return "evidence repeats variable " + std::to_string(v);
            }
            row[v] = (int32_t)x;
        }
        sets.push_back(row);
    }
    return "";
}

std::string query_from_uai(const char *path, const ModelData &m, std::vector<int32_t> &q,
                           bool &parse_error) {
    parse_error = false;
    q.clear();
    std::vector<long long> t;
    std::string err;
    if (!read_ints(path, t, err)) {
        parse_error = err.rfind("cannot open", 0) != 0;
        return err;
    }
    if (t.empty() || t[0] < 0 || (long long)t.size() != 1 + t[0]) {
        parse_error = true;
        return "query file must be \"<nq> v1 ... vq\"";
    }
    std::vector<char> seen(m.nvars, 0);
    for (size_t i = 1; i < t.size(); ++i) {
        if (t[i] < 0 || t[i] >= m.nvars) {
            parse_error = true;
            return "query variable out of range: " + std::to_string(t[i]);
        }
        if (seen[t[i]]) {
            parse_error = true;
            return "query repeats variable " + std::to_string(t[i]);
        }
        seen[t[i]] = 1;
        q.push_back((int32_t)t[i]);
    }
    return "";
}

}  // namespace tn
