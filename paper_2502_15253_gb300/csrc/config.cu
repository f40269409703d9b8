// Model creation from a JSON configuration ([S]: the first component of the framework reads
// a configuration file that names the datasets, their inputs and the parameters with their
// priors). Host code only: a small JSON reader (RFC 8259 values: objects, arrays, numbers,
// strings, true, false, null), the mapping of the configuration onto fit_model_desc, and the
// parameter names, which stay with the model. Parameters are referred to by name (or index);
// a survival-probability entry is either a parameter name or a number (a held constant).
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/fitcore.h"

int fitcore_fail(int code, const std::string &msg);
void fitcore_model_set_names(fit_model *model, const std::vector<std::string> &names);

namespace fitcore {
namespace json {

struct Value {
    enum Kind { Null, Bool, Number, String, Array, Object } kind = Null;
    bool b = false;
    double num = 0.0;
    std::string str;
    std::vector<Value> arr;
    std::vector<std::pair<std::string, Value>> obj;   // in document order

    const Value *get(const std::string &key) const {
        if (kind != Object) return nullptr;
        for (const auto &kv : obj)
            if (kv.first == key) return &kv.second;
        return nullptr;
    }
};

class Parser {
  public:
    explicit Parser(const char *s) : p_(s), s0_(s) {}
    bool parse(Value &v, std::string &err) {
        skip();
        if (!value(v, 0)) {
            err = msg_.empty() ? "malformed JSON" : msg_;
            err += " at offset " + std::to_string(p_ - s0_);
            return false;
        }
        skip();
        if (*p_) {
            err = "trailing characters at offset " + std::to_string(p_ - s0_);
            return false;
        }
        return true;
    }

  private:
    const char *p_, *s0_;
    std::string msg_;
    void skip() {
        while (*p_ == ' ' || *p_ == '\t' || *p_ == '\n' || *p_ == '\r') ++p_;
    }
    bool lit(const char *w) {
        const size_t n = std::strlen(w);
        if (std::strncmp(p_, w, n) != 0) return false;
        p_ += n;
        return true;
    }
    bool value(Value &v, int depth) {
        if (depth > 64) {
            msg_ = "nesting too deep";
            return false;
        }
        skip();
        switch (*p_) {
            case '{': return object(v, depth);
            case '[': return array(v, depth);
            case '"': v.kind = Value::String; return string(v.str);
            case 't': v.kind = Value::Bool; v.b = true; return lit("true");
            case 'f': v.kind = Value::Bool; v.b = false; return lit("false");
            case 'n': v.kind = Value::Null; return lit("null");
            default: return number(v);
        }
    }
    bool number(Value &v) {
        const char *q = p_;
        if (*q == '-') ++q;
        if (!std::isdigit((unsigned char)*q)) {
            msg_ = "expected a value";
            return false;
        }
        char *end = nullptr;
        v.num = std::strtod(p_, &end);
        if (end == p_) return false;
        p_ = end;
        v.kind = Value::Number;
        return true;
    }
    bool hex4(const char *q, unsigned &cp) {
        cp = 0;
        for (int i = 0; i < 4; ++i) {
            const char c = q[i];
            if (!std::isxdigit((unsigned char)c)) {
                msg_ = "bad \\u escape";
                return false;
            }
            cp = cp * 16 + (unsigned)(std::isdigit((unsigned char)c) ? c - '0' : std::tolower((unsigned char)c) - 'a' + 10);
        }
        return true;
    }
    static void utf8(std::string &out, unsigned cp) {
        if (cp < 0x80) {
            out += (char)cp;
        } else if (cp < 0x800) {
            out += (char)(0xC0 | (cp >> 6));
            out += (char)(0x80 | (cp & 0x3F));
        } else if (cp < 0x10000) {
            out += (char)(0xE0 | (cp >> 12));
            out += (char)(0x80 | ((cp >> 6) & 0x3F));
            out += (char)(0x80 | (cp & 0x3F));
        } else {
            out += (char)(0xF0 | (cp >> 18));
            out += (char)(0x80 | ((cp >> 12) & 0x3F));
            out += (char)(0x80 | ((cp >> 6) & 0x3F));
            out += (char)(0x80 | (cp & 0x3F));
        }
    }
    bool string(std::string &out) {
        if (*p_ != '"') return false;
        ++p_;
        out.clear();
        while (*p_ && *p_ != '"') {
            if (*p_ == '\\') {
                ++p_;
                switch (*p_) {
                    case '"': out += '"'; break;
                    case '\\': out += '\\'; break;
                    case '/': out += '/'; break;
                    case 'b': out += '\b'; break;
                    case 'f': out += '\f'; break;
                    case 'n': out += '\n'; break;
                    case 'r': out += '\r'; break;
                    case 't': out += '\t'; break;
                    case 'u': {   // \uXXXX (a surrogate pair for code points above U+FFFF), as UTF-8
                        unsigned cp = 0;
                        if (!hex4(p_ + 1, cp)) return false;
                        p_ += 4;
                        if (cp >= 0xD800 && cp < 0xDC00) {
                            unsigned lo = 0;
                            if (p_[1] != '\\' || p_[2] != 'u' || !hex4(p_ + 3, lo) || lo < 0xDC00 || lo >= 0xE000) {
                                msg_ = "unpaired surrogate";
                                return false;
                            }
                            cp = 0x10000 + ((cp - 0xD800) << 10) + (lo - 0xDC00);
                            p_ += 6;
                        } else if (cp >= 0xDC00 && cp < 0xE000) {
                            msg_ = "unpaired surrogate";
                            return false;
                        }
                        utf8(out, cp);
                        break;
                    }
                    default: msg_ = "bad escape"; return false;
                }
                ++p_;
            } else {
                out += *p_++;
            }
        }
        if (*p_ != '"') {
            msg_ = "unterminated string";
            return false;
        }
        ++p_;
        return true;
    }
    bool array(Value &v, int depth) {
        v.kind = Value::Array;
        ++p_;
        skip();
        if (*p_ == ']') {
            ++p_;
            return true;
        }
        while (true) {
            v.arr.emplace_back();
            if (!value(v.arr.back(), depth + 1)) return false;
            skip();
            if (*p_ == ',') {
                ++p_;
                continue;
            }
            if (*p_ == ']') {
                ++p_;
                return true;
            }
            msg_ = "expected ',' or ']'";
            return false;
        }
    }
    bool object(Value &v, int depth) {
        v.kind = Value::Object;
        ++p_;
        skip();
        if (*p_ == '}') {
            ++p_;
            return true;
        }
        while (true) {
            skip();
            std::string key;
            if (!string(key)) {
                if (msg_.empty()) msg_ = "expected a key";
                return false;
            }
            skip();
            if (*p_ != ':') {
                msg_ = "expected ':'";
                return false;
            }
            ++p_;
            v.obj.emplace_back(key, Value());
            if (!value(v.obj.back().second, depth + 1)) return false;
            skip();
            if (*p_ == ',') {
                ++p_;
                continue;
            }
            if (*p_ == '}') {
                ++p_;
                return true;
            }
            msg_ = "expected ',' or '}'";
            return false;
        }
    }
};

}  // namespace json

namespace {

struct ConfigError {
    std::string msg;
    int code;
};

[[noreturn]] void bad(const std::string &m) { throw ConfigError{m, FIT_ERR_INVALID_CONFIG}; }
[[noreturn]] void not_spd(const std::string &m) { throw ConfigError{m, FIT_ERR_NON_SPD_COV}; }

// Lower Cholesky factor of the symmetric n x n matrix a (row-major); false unless positive definite.
bool cholesky(int n, const std::vector<double> &a, std::vector<double> &l) {
    l.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = a[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= l[(size_t)j * n + k] * l[(size_t)j * n + k];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double r = std::sqrt(d);
        l[(size_t)j * n + j] = r;
        for (int i = j + 1; i < n; ++i) {
            double s = a[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= l[(size_t)i * n + k] * l[(size_t)j * n + k];
            l[(size_t)i * n + j] = s / r;
        }
    }
    return true;
}

// x = (L L^T)^-1 b for one right-hand side, in place
void chol_solve(int n, const std::vector<double> &l, double *x) {
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < i; ++k) x[i] -= l[(size_t)i * n + k] * x[k];
        x[i] /= l[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        for (int k = i + 1; k < n; ++k) x[i] -= l[(size_t)k * n + i] * x[k];
        x[i] /= l[(size_t)i * n + i];
    }
}

// Gaussian prior on b = A theta (A: m x k, m >= k), mean b0, covariance V (m x m), Eq. 6 with
// a linear generalised parametrisation. As a function of theta,
//   (A theta - b0)^T V^-1 (A theta - b0) = (theta - t)^T C^-1 (theta - t) + const
// with C = (A^T V^-1 A)^-1 and t = C A^T V^-1 b0, so the prior is the covariance block C on
// theta with mean t (the constant, the part of b0 no theta reaches, does not depend on theta).
void linear_prior(int m, int k, const std::vector<double> &A, const std::vector<double> &b0,
                  const std::vector<double> &V, const std::string &w, std::vector<double> &C,
                  std::vector<double> &t) {
    std::vector<double> lv, lf;
    if (!cholesky(m, V, lv)) not_spd(w + ".cov: not positive definite");
    std::vector<double> X((size_t)m * k), col(m), wb(b0);   // X = V^-1 A, wb = V^-1 b0
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < m; ++i) col[i] = A[(size_t)i * k + j];
        chol_solve(m, lv, col.data());
        for (int i = 0; i < m; ++i) X[(size_t)i * k + j] = col[i];
    }
    chol_solve(m, lv, wb.data());
    std::vector<double> F((size_t)k * k, 0.0), g(k, 0.0);   // F = A^T V^-1 A, g = A^T V^-1 b0
    for (int a = 0; a < k; ++a) {
        for (int i = 0; i < m; ++i) g[a] += A[(size_t)i * k + a] * wb[i];
        for (int b = 0; b < k; ++b)
            for (int i = 0; i < m; ++i) F[(size_t)a * k + b] += A[(size_t)i * k + a] * X[(size_t)i * k + b];
    }
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < a; ++b) F[(size_t)a * k + b] = F[(size_t)b * k + a] = 0.5 * (F[(size_t)a * k + b] + F[(size_t)b * k + a]);
    if (!cholesky(k, F, lf)) not_spd(w + ".map: A^T V^-1 A is not positive definite (the map does not fix every parameter)");
    C.assign((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j) {
        for (int i = 0; i < k; ++i) col[i] = i == j ? 1.0 : 0.0;
        chol_solve(k, lf, col.data());
        for (int i = 0; i < k; ++i) C[(size_t)i * k + j] = col[i];
    }
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < a; ++b) C[(size_t)a * k + b] = C[(size_t)b * k + a] = 0.5 * (C[(size_t)a * k + b] + C[(size_t)b * k + a]);
    t.assign(k, 0.0);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) t[a] += C[(size_t)a * k + b] * g[b];
}

const json::Value &need(const json::Value &o, const std::string &key, const std::string &where) {
    const json::Value *v = o.get(key);
    if (!v) bad(where + ": missing \"" + key + "\"");
    return *v;
}

double num(const json::Value &v, const std::string &where) {
    if (v.kind != json::Value::Number) bad(where + ": expected a number");
    if (!std::isfinite(v.num)) bad(where + ": number out of range");
    return v.num;
}

int integer(const json::Value &v, const std::string &where) {
    const double x = num(v, where);
    if (x != std::floor(x) || std::fabs(x) > 1e9) bad(where + ": expected an integer");
    return (int)x;
}

const std::vector<json::Value> &arr(const json::Value &v, const std::string &where) {
    if (v.kind != json::Value::Array) bad(where + ": expected an array");
    return v.arr;
}

std::vector<double> numbers(const json::Value &v, const std::string &where) {
    std::vector<double> out;
    for (size_t i = 0; i < arr(v, where).size(); ++i)
        out.push_back(num(v.arr[i], where + "[" + std::to_string(i) + "]"));
    return out;
}

// the parameter table: name -> index
struct Params {
    std::vector<std::string> names;
    std::map<std::string, int> index;
    // a parameter reference: a name, an index, or null (-1: held at its nominal value)
    int ref(const json::Value &v, const std::string &where) const {
        if (v.kind == json::Value::Null) return -1;
        if (v.kind == json::Value::String) {
            auto it = index.find(v.str);
            if (it == index.end()) bad(where + ": unknown parameter \"" + v.str + "\"");
            return it->second;
        }
        const int i = integer(v, where);
        if (i < -1 || i >= (int)names.size()) bad(where + ": parameter index out of range");
        return i;
    }
    std::vector<int> refs(const json::Value &v, const std::string &where) const {
        std::vector<int> out;
        for (size_t i = 0; i < arr(v, where).size(); ++i) out.push_back(ref(v.arr[i], where + "[" + std::to_string(i) + "]"));
        return out;
    }
};

}  // namespace
}  // namespace fitcore

extern "C" int fit_model_create_json(const char *text, fit_model **out) {
    using namespace fitcore;
    if (!text || !out) return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_model_create_json: null argument");
    *out = nullptr;
    json::Value root;
    std::string err;
    if (!json::Parser(text).parse(root, err)) return fitcore_fail(FIT_ERR_INVALID_CONFIG, "fit_model_create_json: " + err);
    try {
        if (root.kind != json::Value::Object) bad("the configuration must be an object");
        // parameters; a group {"namespace": ns, "parameters": [...]} prefixes its members'
        // names with "ns." ([S]: the parameter handling allows several namespaces)
        Params prm;
        std::vector<double> theta0, sigma, scale;
        std::function<void(const json::Value &, const std::string &, const std::string &, int)> add;
        add = [&](const json::Value &list, const std::string &prefix, const std::string &where, int depth) {
            if (depth > 8) bad(where + ": namespaces nested too deep");
            const auto &pl = arr(list, where);
            for (size_t i = 0; i < pl.size(); ++i) {
                const std::string w = where + "[" + std::to_string(i) + "]";
                const json::Value &p = pl[i];
                if (p.kind != json::Value::Object) bad(w + ": expected an object");
                if (const json::Value *ns = p.get("namespace")) {
                    if (ns->kind != json::Value::String || ns->str.empty() || ns->str.find('.') != std::string::npos)
                        bad(w + ".namespace: expected a name without '.'");
                    add(need(p, "parameters", w), prefix + ns->str + ".", w + ".parameters", depth + 1);
                    continue;
                }
                const json::Value &nm = need(p, "name", w);
                if (nm.kind != json::Value::String || nm.str.empty()) bad(w + ".name: expected a string");
                const std::string full = prefix + nm.str;
                if (prm.index.count(full)) bad(w + ": duplicate name \"" + full + "\"");
                prm.index[full] = (int)prm.names.size();
                prm.names.push_back(full);
                theta0.push_back(num(need(p, "value", w), w + ".value"));
                const json::Value *sg = p.get("sigma");
                const json::Value *sc = p.get("scale");
                sigma.push_back(sg ? num(*sg, w + ".sigma") : 0.0);
                scale.push_back(sc ? num(*sc, w + ".scale") : 0.0);
            }
        };
        add(need(root, "parameters", "config"), "", "parameters", 0);
        const int P = (int)prm.names.size();
        // covariance blocks
        std::vector<int> cov_size, cov_idx;
        std::vector<double> cov;
        if (const json::Value *cb = root.get("covariances")) {
            for (size_t b = 0; b < arr(*cb, "covariances").size(); ++b) {
                const std::string w = "covariances[" + std::to_string(b) + "]";
                const json::Value &blk = cb->arr[b];
                const std::vector<int> idx = prm.refs(need(blk, "params", w), w + ".params");
                const int k = (int)idx.size();
                const json::Value *mp = blk.get("map");
                const int m = mp ? (int)arr(*mp, w + ".map").size() : k;
                std::vector<double> V;
                const auto &rows = arr(need(blk, "cov", w), w + ".cov");
                if ((int)rows.size() != m) bad(w + ".cov: expected " + std::to_string(m) + " rows");
                for (size_t r = 0; r < rows.size(); ++r) {
                    const std::vector<double> row = numbers(rows[r], w + ".cov[" + std::to_string(r) + "]");
                    if ((int)row.size() != m) bad(w + ".cov: rows must be square");
                    V.insert(V.end(), row.begin(), row.end());
                }
                for (int i : idx)
                    if (i < 0) bad(w + ".params: null is not a parameter");
                if (mp) {   // prior on b = A theta with mean b0: the equivalent block on theta
                    if (m < k) bad(w + ".map: fewer rows than parameters");
                    std::vector<double> A;
                    for (int r = 0; r < m; ++r) {
                        const std::vector<double> row = numbers(mp->arr[r], w + ".map[" + std::to_string(r) + "]");
                        if ((int)row.size() != k) bad(w + ".map: rows need one entry per parameter");
                        A.insert(A.end(), row.begin(), row.end());
                    }
                    const std::vector<double> b0 = numbers(need(blk, "mean", w), w + ".mean");
                    if ((int)b0.size() != m) bad(w + ".mean: one entry per map row");
                    std::vector<double> Cb, tb;
                    linear_prior(m, k, A, b0, V, w, Cb, tb);
                    for (int i = 0; i < k; ++i) theta0[idx[i]] = tb[i];
                    V.swap(Cb);
                }
                cov.insert(cov.end(), V.begin(), V.end());
                for (int i : idx) cov_idx.push_back(i);
                cov_size.push_back((int)idx.size());
            }
        }
        // survival
        const json::Value &osc = need(root, "oscillation", "config");
        const json::Value &formula = need(osc, "formula", "oscillation");
        int mode = -1;
        if (formula.kind == json::Value::String) {
            if (formula.str == "eq1") mode = FIT_OSC_EQ1;
            else if (formula.str == "vacuum3") mode = FIT_OSC_VACUUM3;
            else if (formula.str == "sterile4") mode = FIT_OSC_STERILE4;
        }
        if (mode < 0) bad("oscillation.formula: one of \"eq1\", \"vacuum3\", \"sterile4\"");
        const int n_osc = mode == FIT_OSC_STERILE4 ? 6 : 4;
        const auto &op = arr(need(osc, "params", "oscillation"), "oscillation.params");
        if ((int)op.size() != n_osc) bad("oscillation.params: expected " + std::to_string(n_osc) + " entries");
        fit_model_desc d;
        std::memset(&d, 0, sizeof(d));
        d.osc_mode = mode;
        for (int i = 0; i < 6; ++i) d.osc_idx[i] = -1;
        for (int i = 0; i < n_osc; ++i) {
            const std::string w = "oscillation.params[" + std::to_string(i) + "]";
            if (op[i].kind == json::Value::String) {   // a fit parameter, by name
                d.osc_idx[i] = prm.ref(op[i], w);
                d.osc_val[i] = theta0[d.osc_idx[i]];
            } else {                                    // a held constant
                d.osc_val[i] = num(op[i], w);
            }
        }
        // grid, energy correction
        const json::Value &grid = need(root, "true_grid", "config");
        d.n_true = integer(need(grid, "bins", "true_grid"), "true_grid.bins");
        d.e_lo = num(need(grid, "e_lo", "true_grid"), "true_grid.e_lo");
        d.e_hi = num(need(grid, "e_hi", "true_grid"), "true_grid.e_hi");
        d.remap_mode = FIT_REMAP_OVERLAP;
        if (const json::Value *ec = root.get("energy_correction")) {
            if (ec->kind != json::Value::String || (ec->str != "overlap" && ec->str != "spline"))
                bad("energy_correction: \"overlap\" or \"spline\"");
            d.remap_mode = ec->str == "spline" ? FIT_REMAP_SPLINE : FIT_REMAP_OVERLAP;
        }
        const int Nt = d.n_true;
        // cores
        const std::vector<int> cpw = prm.refs(need(root, "core_powers", "config"), "core_powers");
        // detectors
        std::vector<int> det_n_reco;
        std::vector<double> det_resp;
        std::map<std::string, int> det_by_name;
        const auto &dl = arr(need(root, "detectors", "config"), "detectors");
        for (size_t k = 0; k < dl.size(); ++k) {
            const std::string w = "detectors[" + std::to_string(k) + "]";
            if (const json::Value *nm = dl[k].get("name"))
                if (nm->kind == json::Value::String) det_by_name[nm->str] = (int)k;
            const auto &rows = arr(need(dl[k], "response", w), w + ".response");
            for (size_t r = 0; r < rows.size(); ++r) {
                const std::vector<double> row = numbers(rows[r], w + ".response[" + std::to_string(r) + "]");
                if ((int)row.size() != Nt) bad(w + ".response: rows need true_grid.bins entries");
                det_resp.insert(det_resp.end(), row.begin(), row.end());
            }
            det_n_reco.push_back((int)rows.size());
        }
        // datasets
        std::vector<int> ds_det, ds_norm, ds_eff, ds_esc, ds_shape;
        std::vector<double> ds_t, ds_L, ds_w;
        std::vector<int> bkg_ds, bkg_rate, bkg_shape;
        std::vector<double> bkg_tmpl;
        const int C = (int)cpw.size();
        const auto &dsl = arr(need(root, "datasets", "config"), "datasets");
        for (size_t k = 0; k < dsl.size(); ++k) {
            const std::string w = "datasets[" + std::to_string(k) + "]";
            const json::Value &ds = dsl[k];
            const json::Value &dv = need(ds, "detector", w);
            int det = -1;
            if (dv.kind == json::Value::String) {
                auto it = det_by_name.find(dv.str);
                if (it == det_by_name.end()) bad(w + ".detector: unknown detector \"" + dv.str + "\"");
                det = it->second;
            } else {
                det = integer(dv, w + ".detector");
            }
            if (det < 0 || det >= (int)det_n_reco.size()) bad(w + ".detector: out of range");
            ds_det.push_back(det);
            const std::vector<double> t = numbers(need(ds, "t", w), w + ".t");
            if ((int)t.size() != Nt) bad(w + ".t: expected true_grid.bins entries");
            ds_t.insert(ds_t.end(), t.begin(), t.end());
            const std::vector<double> L = numbers(need(ds, "baseline", w), w + ".baseline");
            const std::vector<double> cw = numbers(need(ds, "weight", w), w + ".weight");
            if ((int)L.size() != C || (int)cw.size() != C) bad(w + ": baseline and weight need one entry per core");
            ds_L.insert(ds_L.end(), L.begin(), L.end());
            ds_w.insert(ds_w.end(), cw.begin(), cw.end());
            const json::Value *nv = ds.get("norm");
            const json::Value *ev = ds.get("efficiency");
            ds_norm.push_back(nv ? prm.ref(*nv, w + ".norm") : -1);
            ds_eff.push_back(ev ? prm.ref(*ev, w + ".efficiency") : -1);
            std::vector<int> esc(3, -1);
            if (const json::Value *e = ds.get("escale")) {
                esc = prm.refs(*e, w + ".escale");
                if (esc.size() != 3) bad(w + ".escale: three entries (a0, a1, a2)");
            }
            ds_esc.insert(ds_esc.end(), esc.begin(), esc.end());
            std::vector<int> sh(Nt, -1);
            if (const json::Value *s = ds.get("shape")) {
                sh = prm.refs(*s, w + ".shape");
                if ((int)sh.size() != Nt) bad(w + ".shape: expected true_grid.bins entries");
            }
            ds_shape.insert(ds_shape.end(), sh.begin(), sh.end());
            // backgrounds of this dataset, in reco space (Eq. 8)
            if (const json::Value *bl = ds.get("backgrounds")) {
                const int nr = det_n_reco[det];
                for (size_t j = 0; j < arr(*bl, w + ".backgrounds").size(); ++j) {
                    const std::string wb = w + ".backgrounds[" + std::to_string(j) + "]";
                    const json::Value &b = bl->arr[j];
                    const std::vector<double> tm = numbers(need(b, "template", wb), wb + ".template");
                    if ((int)tm.size() != nr) bad(wb + ".template: one entry per reco bin of the detector");
                    std::vector<int> bsh(nr, -1);
                    if (const json::Value *s2 = b.get("shape")) {
                        bsh = prm.refs(*s2, wb + ".shape");
                        if ((int)bsh.size() != nr) bad(wb + ".shape: one entry per reco bin");
                    }
                    const json::Value *rv = b.get("rate");
                    bkg_ds.push_back((int)k);
                    bkg_rate.push_back(rv ? prm.ref(*rv, wb + ".rate") : -1);
                    bkg_tmpl.insert(bkg_tmpl.end(), tm.begin(), tm.end());
                    bkg_shape.insert(bkg_shape.end(), bsh.begin(), bsh.end());
                }
            }
        }
        // the description (arrays live until fit_model_create returns)
        const std::vector<double> one(1, 0.0);
        const std::vector<int> ione(1, 0);
        d.n_params = P;
        d.theta0 = theta0.data();
        d.prior_sigma = sigma.data();
        d.scale = scale.data();
        d.n_cov = (int)cov_size.size();
        d.cov_size = cov_size.empty() ? ione.data() : cov_size.data();
        d.cov_idx = cov_idx.empty() ? ione.data() : cov_idx.data();
        d.cov = cov.empty() ? one.data() : cov.data();
        d.n_cores = C;
        d.core_power_idx = cpw.empty() ? ione.data() : cpw.data();
        d.n_det = (int)det_n_reco.size();
        d.det_n_reco = det_n_reco.empty() ? ione.data() : det_n_reco.data();
        d.det_response = det_resp.empty() ? one.data() : det_resp.data();
        d.n_ds = (int)ds_det.size();
        d.ds_det = ds_det.empty() ? ione.data() : ds_det.data();
        d.ds_t = ds_t.empty() ? one.data() : ds_t.data();
        d.ds_baseline = ds_L.empty() ? one.data() : ds_L.data();
        d.ds_weight = ds_w.empty() ? one.data() : ds_w.data();
        d.ds_norm_idx = ds_norm.empty() ? ione.data() : ds_norm.data();
        d.ds_eff_idx = ds_eff.empty() ? ione.data() : ds_eff.data();
        d.ds_escale_idx = ds_esc.empty() ? ione.data() : ds_esc.data();
        d.ds_shape_idx = ds_shape.empty() ? ione.data() : ds_shape.data();
        d.n_bkg = (int)bkg_ds.size();
        d.bkg_ds = bkg_ds.empty() ? ione.data() : bkg_ds.data();
        d.bkg_template = bkg_tmpl.empty() ? one.data() : bkg_tmpl.data();
        d.bkg_rate_idx = bkg_rate.empty() ? ione.data() : bkg_rate.data();
        d.bkg_shape_idx = bkg_shape.empty() ? ione.data() : bkg_shape.data();
        fit_model *m = nullptr;
        const int rc = fit_model_create(&d, &m);
        if (rc != FIT_OK) return rc;
        fitcore_model_set_names(m, prm.names);
        *out = m;
        return FIT_OK;
    } catch (const ConfigError &e) {
        return fitcore_fail(e.code, "fit_model_create_json: " + e.msg);
    }
}

// ---- best-fit output as JSON ([S]: the third component writes the converged fit to a JSON
// file, the interface to the rest of an analysis chain) --------------------------------------
namespace {

const char *status_name(int s) {
    static const char *k[] = {"converged", "maxiter", "linesearch_fail", "nonfinite",
                              "mu_nonpositive", "escale_nonmonotone", "timeout", "stalled"};
    return s >= 0 && s < 8 ? k[s] : "unknown";
}

void put_number(std::string &o, double x) {
    if (!std::isfinite(x)) {   // JSON has no inf / nan
        o += "null";
        return;
    }
    char b[32];
    std::snprintf(b, sizeof(b), "%.17g", x);
    o += b;
}

void put_string(std::string &o, const char *s) {
    o += '"';
    for (; *s; ++s) {
        const unsigned char c = (unsigned char)*s;
        if (c == '"' || c == '\\') {
            o += '\\';
            o += (char)c;
        } else if (c < 0x20) {
            char b[8];
            std::snprintf(b, sizeof(b), "\\u%04x", c);
            o += b;
        } else {
            o += (char)c;
        }
    }
    o += '"';
}

}  // namespace

extern "C" int fit_result_json(const fit_model *model, const double *best, const fit_result *res,
                               char *buf, size_t buf_len, size_t *needed) {
    if (!model || !best || !res || !needed) return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_result_json: null argument");
    fit_model_info_t info;
    const int rc = fit_model_info(model, &info);
    if (rc != FIT_OK) return rc;
    std::string o = "{\"nll_min\": ";
    put_number(o, res->nll_min);
    o += ", \"edm\": ";
    put_number(o, res->edm);
    o += ", \"iters\": " + std::to_string(res->iters) + ", \"n_evals\": " + std::to_string(res->n_evals);
    o += ", \"status\": ";
    put_string(o, status_name(res->status));
    o += ", \"params\": {";
    for (int i = 0; i < info.n_params; ++i) {
        if (i) o += ", ";
        const char *nm = fit_model_param_name(model, i);
        put_string(o, nm ? nm : ("p" + std::to_string(i)).c_str());
        o += ": ";
        put_number(o, best[i]);
    }
    o += "}}";
    *needed = o.size() + 1;
    if (!buf) return FIT_OK;
    if (buf_len < o.size() + 1) return fitcore_fail(FIT_ERR_INVALID_ARG, "fit_result_json: buffer too small");
    std::memcpy(buf, o.c_str(), o.size() + 1);
    return FIT_OK;
}
