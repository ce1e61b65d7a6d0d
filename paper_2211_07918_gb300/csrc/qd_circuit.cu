// Circuit-level host code of libqudit: the QuDiet QASM front end (Sec. 4),
// the Toffoli decomposition through an elevated carrier level (Sec. 3.4) and
// the logarithmic-depth multi-controlled Toffoli through |d>-level controls
// (Sec. 2.1.2, Fig. 1), and ket labels of basis states (Sec. 3.8).  Nothing
// here touches the device: the gates it produces run through the same
// planner and kernels as any other gate list.
#include <cctype>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qudit.h"

namespace qd {
int set_last_error(int code, const char *msg);  // qd_api.cu
}

namespace {

int circ_fail(int code, const std::string &msg) { return qd::set_last_error(code, msg.c_str()); }

qd_gate blank_gate(int32_t kind) {
    qd_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = kind;
    return g;
}

// X^{d_t}_{+shift} on t when every control holds its level.
qd_gate shift_gate(int32_t t, int32_t shift, const int32_t *controls, const int32_t *levels, int32_t nc) {
    qd_gate g = blank_gate(QD_GATE_X);
    g.k = 1;
    g.targets[0] = t;
    g.param = shift;
    g.nc = nc;
    for (int i = 0; i < nc; ++i) {
        g.controls[i] = controls[i];
        g.ctrl_levels[i] = levels[i];
    }
    return g;
}

bool qudit_ok(const int32_t *dims, int32_t n, int32_t q) { return q >= 0 && q < n && dims[q] >= 2; }

// ---------------------------------------------------------------- QASM lexer

std::string lower(std::string s) {
    for (char &c : s) c = (char)std::tolower((unsigned char)c);
    return s;
}

// Split a line into tokens at whitespace; '(' and ')' are tokens of their own;
// '#' or "//" starts a comment.
std::vector<std::string> tokens_of(const std::string &line) {
    std::vector<std::string> out;
    std::string cur;
    auto flush = [&] {
        if (!cur.empty()) out.push_back(cur);
        cur.clear();
    };
    for (size_t i = 0; i < line.size(); ++i) {
        const char c = line[i];
        if (c == '#' || (c == '/' && i + 1 < line.size() && line[i + 1] == '/')) break;
        if (std::isspace((unsigned char)c)) {
            flush();
        } else if (c == '(' || c == ')' || c == ',') {
            flush();
            if (c != ',') out.push_back(std::string(1, c));
        } else {
            cur.push_back(c);
        }
    }
    flush();
    return out;
}

bool parse_int(const std::string &s, long &v) {
    if (s.empty()) return false;
    char *end = nullptr;
    v = std::strtol(s.c_str(), &end, 10);
    return end && *end == '\0';
}

}  // namespace

extern "C" {

// QuDiet QASM (Sec. 4): ".qudit n", then n declarations "qudit NAME (d)" in
// qudit order, then ".begin", gate lines, ".end".  Gate lines: "X q [a]"
// (X^d_{+a}, a = 1 if absent), "Z q [p]" (Z_d^p), "H q" (F_d), "CX c t [a]"
// (X^{d_t}_{+a} on t when c holds d_c - 1).  Names are case-insensitive.
int qd_qasm_parse(const char *text, int32_t *dims, int32_t dims_cap, int32_t *n_out, qd_gate *gates,
                  int32_t gates_cap, int32_t *ngates_out, int32_t *error_line) {
    if (error_line) *error_line = 0;
    if (!text || !n_out || !ngates_out) return circ_fail(QD_ERR_ARG, "qasm: null text or count pointer");
    std::vector<std::string> names;
    std::vector<int32_t> ds;
    std::vector<qd_gate> gs;
    long declared = -1;
    int section = 0;  // 0: header, 1: inside .begin/.end, 2: after .end
    int line_no = 0;
    const char *p = text;
    auto fail_at = [&](int code, const std::string &msg) {
        if (error_line) *error_line = line_no;
        return circ_fail(code, "qasm line " + std::to_string(line_no) + ": " + msg);
    };
    auto qudit_index = [&](const std::string &name) -> int {
        const std::string l = lower(name);
        for (size_t i = 0; i < names.size(); ++i)
            if (names[i] == l) return (int)i;
        return -1;
    };
    while (*p) {
        const char *e = std::strchr(p, '\n');
        const std::string line = e ? std::string(p, e - p) : std::string(p);
        p = e ? e + 1 : p + line.size();
        ++line_no;
        const std::vector<std::string> tk = tokens_of(line);
        if (tk.empty()) continue;
        const std::string op = lower(tk[0]);
        if (op == ".qudit") {
            if (section != 0 || declared >= 0) return fail_at(QD_ERR_ARG, ".qudit must appear once, first");
            long v = 0;
            if (tk.size() != 2 || !parse_int(tk[1], v) || v < 1 || v > QD_MAX_QUDITS)
                return fail_at(QD_ERR_ARG, ".qudit needs a count in [1, 48]");
            declared = v;
            continue;
        }
        if (op == "qudit") {
            if (section != 0 || declared < 0) return fail_at(QD_ERR_ARG, "qudit declarations follow .qudit, before .begin");
            long d = 0;
            if (tk.size() != 5 || tk[2] != "(" || tk[4] != ")" || !parse_int(tk[3], d))
                return fail_at(QD_ERR_ARG, "declaration must read: qudit NAME (d)");
            if (d < 2 || d > 64) return fail_at(QD_ERR_DIM, "qudit dimension must be in [2, 64]");
            if (qudit_index(tk[1]) >= 0) return fail_at(QD_ERR_ARG, "qudit " + tk[1] + " declared twice");
            if ((long)names.size() >= declared) return fail_at(QD_ERR_ARG, "more declarations than .qudit states");
            names.push_back(lower(tk[1]));
            ds.push_back((int32_t)d);
            continue;
        }
        if (op == ".begin") {
            if (section != 0 || (long)names.size() != declared || declared < 1)
                return fail_at(QD_ERR_ARG, ".begin needs every qudit of .qudit declared first");
            section = 1;
            continue;
        }
        if (op == ".end") {
            if (section != 1) return fail_at(QD_ERR_ARG, ".end without .begin");
            section = 2;
            continue;
        }
        if (section != 1) return fail_at(QD_ERR_ARG, "gate outside .begin/.end: " + tk[0]);
        const int nq = (int)names.size();
        auto operand = [&](size_t i, int &q) -> int {
            q = qudit_index(tk[i]);
            if (q < 0) return fail_at(QD_ERR_ARG, "unknown qudit " + tk[i]);
            return QD_OK;
        };
        if (op == "x" || op == "z" || op == "h") {
            const size_t want_max = op == "h" ? 2 : 3;
            if (tk.size() < 2 || tk.size() > want_max) return fail_at(QD_ERR_ARG, "bad operand count for " + tk[0]);
            int q = -1;
            if (int rc = operand(1, q)) return rc;
            long a = 1;
            if (tk.size() == 3 && !parse_int(tk[2], a)) return fail_at(QD_ERR_ARG, "bad integer " + tk[2]);
            qd_gate g = blank_gate(op == "x" ? QD_GATE_X : op == "z" ? QD_GATE_Z : QD_GATE_H);
            g.k = 1;
            g.targets[0] = q;
            if (op == "x") {
                if (a < 1 || a >= ds[q]) return fail_at(QD_ERR_ARG, "X shift must be in [1, d-1]");
                g.param = (int32_t)a;
            } else if (op == "z") {
                g.param = (int32_t)a;
            }
            gs.push_back(g);
            (void)nq;
            continue;
        }
        if (op == "cx") {
            if (tk.size() < 3 || tk.size() > 4) return fail_at(QD_ERR_ARG, "CX needs control, target [, shift]");
            int c = -1, t = -1;
            if (int rc = operand(1, c)) return rc;
            if (int rc = operand(2, t)) return rc;
            if (c == t) return fail_at(QD_ERR_OVERLAP, "CX control and target are the same qudit");
            long a = 1;
            if (tk.size() == 4 && !parse_int(tk[3], a)) return fail_at(QD_ERR_ARG, "bad integer " + tk[3]);
            if (a < 1 || a >= ds[t]) return fail_at(QD_ERR_ARG, "CX shift must be in [1, d_t - 1]");
            const int32_t lv = -1;
            gs.push_back(shift_gate(t, (int32_t)a, &c, &lv, 1));
            continue;
        }
        return fail_at(QD_ERR_ARG, "unknown gate " + tk[0]);
    }
    if (declared < 0) return circ_fail(QD_ERR_ARG, "qasm: no .qudit line");
    if (section == 0) return circ_fail(QD_ERR_ARG, "qasm: no .begin line");
    if (section == 1) return circ_fail(QD_ERR_ARG, "qasm: .begin without .end");
    *n_out = (int32_t)ds.size();
    *ngates_out = (int32_t)gs.size();
    if ((dims && dims_cap < (int32_t)ds.size()) || (gates && gates_cap < (int32_t)gs.size()))
        return circ_fail(QD_ERR_OOM, "qasm: output arrays too small (counts written)");
    if (dims) std::memcpy(dims, ds.data(), ds.size() * sizeof(int32_t));
    if (gates && !gs.empty()) std::memcpy(gates, gs.data(), gs.size() * sizeof(qd_gate));
    return QD_OK;
}

// Toffoli through an elevated carrier (Sec. 3.4): CX_{+1}(c1 -> carrier),
// CX_{+shift}(carrier -> t), CX_{+(d_carrier - 1)}(c1 -> carrier), every
// control firing on its top level d - 1.  The carrier's logical levels are
// [0, d_carrier - 2]; the first CX raises its top logical level to the
// elevated level d_carrier - 1, which only that case reaches.
int qd_toffoli_gates(const int32_t *dims, int32_t n, int32_t c1, int32_t carrier, int32_t t, int32_t shift,
                     qd_gate *out) {
    if (!dims || !out) return circ_fail(QD_ERR_ARG, "toffoli: null pointer");
    if (!qudit_ok(dims, n, c1) || !qudit_ok(dims, n, carrier) || !qudit_ok(dims, n, t))
        return circ_fail(QD_ERR_ARG, "toffoli: qudit index out of range");
    if (c1 == carrier || c1 == t || carrier == t) return circ_fail(QD_ERR_OVERLAP, "toffoli: qudits must differ");
    if (dims[carrier] < 3) return circ_fail(QD_ERR_DIM, "toffoli: the carrier needs a free level (dimension >= 3)");
    if (shift < 1 || shift >= dims[t]) return circ_fail(QD_ERR_ARG, "toffoli: shift must be in [1, d_t - 1]");
    const int32_t top1 = dims[c1] - 1, topc = dims[carrier] - 1;
    out[0] = shift_gate(carrier, 1, &c1, &top1, 1);
    out[1] = shift_gate(t, shift, &carrier, &topc, 1);
    out[2] = shift_gate(carrier, dims[carrier] - 1, &c1, &top1, 1);
    return QD_OK;
}

// Logarithmic-depth multi-controlled Toffoli (Sec. 2.1.2, Fig. 1).  The
// controls form a balanced binary tree (heap order: control i has children
// 2i+1 and 2i+2).  Control q is active at level l_q (ctrl_levels, NULL or -1:
// d_q - 2) and every control with children needs the free level l_q + 1 <
// d_q, its "|d>" level.  Compute: deepest level first, each inner node v is
// shifted +1 under its children, each child firing on l_u if it is a leaf
// and on its elevated level l_u + 1 otherwise, so v reaches l_v + 1 iff every
// control of its subtree is active (no other value of v reaches it, since the
// logical values of v are <= l_v).  Then X^{d_t}_{+shift} on t under the
// root, and the compute gates undone in reverse order (shift d_v - 1 = -1).
// Gates on one tree level act on disjoint qudits, so the depth is
// 2 floor(log2 nc) + 1.
int qd_mct_tree_gates(const int32_t *dims, int32_t n, const int32_t *controls, const int32_t *ctrl_levels,
                      int32_t nc, int32_t t, int32_t shift, qd_gate *out, int32_t cap, int32_t *count,
                      int32_t *depth) {
    if (!dims || !controls || !count) return circ_fail(QD_ERR_ARG, "mct tree: null pointer");
    if (nc < 1 || nc > 64) return circ_fail(QD_ERR_ARG, "mct tree: control count must be in [1, 64]");
    if (!qudit_ok(dims, n, t)) return circ_fail(QD_ERR_ARG, "mct tree: target out of range");
    if (shift < 1 || shift >= dims[t]) return circ_fail(QD_ERR_ARG, "mct tree: shift must be in [1, d_t - 1]");
    std::vector<int32_t> lv(nc);
    for (int i = 0; i < nc; ++i) {
        const int32_t q = controls[i];
        if (!qudit_ok(dims, n, q)) return circ_fail(QD_ERR_ARG, "mct tree: control out of range");
        if (q == t) return circ_fail(QD_ERR_OVERLAP, "mct tree: a control is the target");
        for (int j = 0; j < i; ++j)
            if (controls[j] == q) return circ_fail(QD_ERR_OVERLAP, "mct tree: repeated control");
        lv[i] = (ctrl_levels && ctrl_levels[i] >= 0) ? ctrl_levels[i] : dims[q] - 2;
        const bool inner = 2 * i + 1 < nc;
        if (lv[i] < 0 || lv[i] >= dims[q]) return circ_fail(QD_ERR_ARG, "mct tree: control level out of range");
        if (inner && lv[i] + 1 >= dims[q])
            return circ_fail(QD_ERR_DIM, "mct tree: an inner control needs a free level above its active level");
    }
    std::vector<qd_gate> comp;
    int levels = 0;
    while ((1 << (levels + 1)) - 1 < nc) ++levels;  // tree depth (root at depth 0)
    for (int lvl = levels - 1; lvl >= 0; --lvl) {
        for (int v = (1 << lvl) - 1; v < (1 << (lvl + 1)) - 1 && v < nc; ++v) {
            int32_t cs[2], cl[2];
            int m = 0;
            for (int u = 2 * v + 1; u <= 2 * v + 2 && u < nc; ++u) {
                cs[m] = controls[u];
                cl[m] = (2 * u + 1 < nc) ? lv[u] + 1 : lv[u];
                ++m;
            }
            if (m > 0) comp.push_back(shift_gate(controls[v], 1, cs, cl, m));
        }
    }
    std::vector<qd_gate> all = comp;
    const int32_t root_level = nc > 1 ? lv[0] + 1 : lv[0];
    all.push_back(shift_gate(t, shift, &controls[0], &root_level, 1));
    for (int i = (int)comp.size() - 1; i >= 0; --i) {
        qd_gate g = comp[i];
        g.param = dims[g.targets[0]] - 1;
        all.push_back(g);
    }
    *count = (int32_t)all.size();
    if (depth) *depth = 2 * levels + 1;
    if (out) {
        if (cap < (int32_t)all.size()) return circ_fail(QD_ERR_OOM, "mct tree: output array too small (count written)");
        std::memcpy(out, all.data(), all.size() * sizeof(qd_gate));
    }
    return QD_OK;
}

// Ket label of basis index i (Sec. 3.8 OutputType.print; Sec. 3.9 prints
// |120> for digits x_0 = 1, x_1 = 2, x_2 = 0): digits qudit 0 first, each in
// decimal, separated by commas when some dimension exceeds 10.
int qd_ket_label(const int32_t *dims, int32_t n, int64_t index, char *buf, int32_t cap) {
    if (!dims || !buf || n < 1 || cap < 1) return circ_fail(QD_ERR_ARG, "ket label: bad arguments");
    bool wide = false;
    int64_t N = 1;
    for (int q = 0; q < n; ++q) {
        if (dims[q] < 2 || dims[q] > 64) return circ_fail(QD_ERR_DIM, "ket label: dimension out of range");
        wide = wide || dims[q] > 10;
        N *= dims[q];
    }
    if (index < 0 || index >= N) return circ_fail(QD_ERR_ARG, "ket label: index out of range");
    std::string s = "|";
    int64_t r = index;
    for (int q = 0; q < n; ++q) {
        if (q > 0 && wide) s += ",";
        s += std::to_string(r % dims[q]);
        r /= dims[q];
    }
    s += ">";
    if ((int32_t)s.size() + 1 > cap) return circ_fail(QD_ERR_OOM, "ket label: buffer too small");
    std::memcpy(buf, s.c_str(), s.size() + 1);
    return QD_OK;
}

}  // extern "C"
