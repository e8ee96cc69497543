// OpenQASM 2.0 import (unitary subset) into qs_gate records.
//
// Program structure: statements `OPENQASM 2.0;`, `include "qelib1.inc";`,
// `qreg r[k];`, `creg c[k];`, `gate g(params) args { body }`, `opaque ...;`,
// `barrier ...;` (skipped), `measure a -> c;` (only after the last unitary
// gate: the state before the measurements is the result), and gate calls.
// Registers are laid end to end in declaration order: the first qreg holds
// qubits 0..k-1, the next one continues from k, and so on.
//
// Gate calls resolve in this order: a `gate` definition of that name in the
// program (inlined with its parameters and arguments bound, recursively,
// using only gates defined before it), else the library's own gates under
// their OpenQASM names (the primitives U and CX and the standard-library
// names: cx -> CX, cu1 / cp -> CPHASE, u1 / p -> P, ...; cu3 as the exact
// two-CX construction of controlled-U3 from RZ, RY, CX and P; c3x / c4x as
// exact ancilla-free phase polynomials of CX and P between H; sxdg as SX^3),
// else an error.
// A call whose arguments are whole registers applies the gate once per index
// (all register arguments of one call have the same size; single-qubit
// arguments are repeated).
//
// Angle expressions: decimal and exponent literals, pi, the gate's
// parameters, + - * / ^, unary minus, parentheses and sin, cos, tan, exp, ln,
// sqrt; evaluated in double precision.
#include "qs_qasm.h"

#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>

namespace qs {
namespace {

struct Tok {
    enum Kind { ID, NUM, STR, SYM, END } kind = END;
    std::string s;   // identifier, string contents or symbol text
    double v = 0;    // NUM
    int line = 0;
};

struct ParseError {
    qs_status st;
    std::string msg;
};

[[noreturn]] void bad(int line, const std::string &m, qs_status st = QS_ERR_INVALID_ARG) {
    throw ParseError{st, "line " + std::to_string(line) + ": " + m};
}

std::vector<Tok> lex(const char *src) {
    std::vector<Tok> out;
    int line = 1;
    const char *p = src;
    while (*p) {
        const char c = *p;
        if (c == '\n') {
            ++line;
            ++p;
            continue;
        }
        if (std::isspace((unsigned char)c)) {
            ++p;
            continue;
        }
        if (c == '/' && p[1] == '/') {
            while (*p && *p != '\n') ++p;
            continue;
        }
        if (c == '/' && p[1] == '*') {
            p += 2;
            while (*p && !(p[0] == '*' && p[1] == '/')) {
                if (*p == '\n') ++line;
                ++p;
            }
            if (!*p) bad(line, "unterminated comment");
            p += 2;
            continue;
        }
        Tok t;
        t.line = line;
        if (std::isalpha((unsigned char)c) || c == '_') {
            const char *q = p;
            while (std::isalnum((unsigned char)*q) || *q == '_') ++q;
            t.kind = Tok::ID;
            t.s.assign(p, q);
            p = q;
        } else if (std::isdigit((unsigned char)c) || (c == '.' && std::isdigit((unsigned char)p[1]))) {
            char *q = nullptr;
            t.kind = Tok::NUM;
            t.v = std::strtod(p, &q);
            t.s.assign(p, static_cast<const char *>(q));
            p = q;
        } else if (c == '"') {
            const char *q = p + 1;
            while (*q && *q != '"' && *q != '\n') ++q;
            if (*q != '"') bad(line, "unterminated string");
            t.kind = Tok::STR;
            t.s.assign(p + 1, q);
            p = q + 1;
        } else if (c == '-' && p[1] == '>') {
            t.kind = Tok::SYM;
            t.s = "->";
            p += 2;
        } else if (c == '=' && p[1] == '=') {
            t.kind = Tok::SYM;
            t.s = "==";
            p += 2;
        } else if (std::strchr(";,()[]{}+-*/^", c)) {
            t.kind = Tok::SYM;
            t.s.assign(1, c);
            ++p;
        } else {
            bad(line, std::string("unexpected character '") + c + "'");
        }
        out.push_back(t);
    }
    Tok e;
    e.kind = Tok::END;
    e.line = line;
    out.push_back(e);
    return out;
}

// token cursor over [pos, end)
struct Cursor {
    const std::vector<Tok> *t;
    size_t pos, end;
    const Tok &peek() const { return (*t)[pos < end ? pos : end]; }
    const Tok &next() {
        const Tok &k = peek();
        if (pos < end) ++pos;
        return k;
    }
    bool at_end() const { return pos >= end || (*t)[pos].kind == Tok::END; }
    bool is_sym(const char *s) const { return peek().kind == Tok::SYM && peek().s == s; }
    bool is_id(const char *s) const { return peek().kind == Tok::ID && peek().s == s; }
    void expect_sym(const char *s) {
        if (!is_sym(s)) bad(peek().line, std::string("expected '") + s + "'" + got());
        next();
    }
    std::string expect_id(const char *what) {
        if (peek().kind != Tok::ID) bad(peek().line, std::string("expected ") + what + got());
        return next().s;
    }
    long expect_int(const char *what) {
        const Tok &k = peek();
        if (k.kind != Tok::NUM || k.s.find_first_not_of("0123456789") != std::string::npos)
            bad(k.line, std::string("expected ") + what + got());
        next();
        return std::strtol(k.s.c_str(), nullptr, 10);
    }
    std::string got() const {
        const Tok &k = peek();
        if (k.kind == Tok::END) return " before the end of the program";
        return " at '" + k.s + "'";
    }
};

// expression grammar: sum := term (('+'|'-') term)*; term := unary (('*'|'/') unary)*;
// unary := '-' unary | power; power := atom ('^' unary)?
constexpr int kMaxExprDepth = 200;   // nesting of parentheses, signs and powers

class Expr {
  public:
    Expr(Cursor &c, const std::map<std::string, double> &env) : c_(c), env_(env) {}
    double sum() {
        Depth guard(this);
        double v = term();
        while (c_.is_sym("+") || c_.is_sym("-")) {
            const bool plus = c_.next().s == "+";
            const double r = term();
            v = plus ? v + r : v - r;
        }
        return v;
    }

  private:
    Cursor &c_;
    const std::map<std::string, double> &env_;
    int depth_ = 0;
    struct Depth {
        Expr *e;
        explicit Depth(Expr *x) : e(x) {
            if (++e->depth_ > kMaxExprDepth) bad(e->c_.peek().line, "expression nested too deeply", QS_ERR_UNSUPPORTED);
        }
        ~Depth() { --e->depth_; }
    };
    double term() {
        double v = unary();
        while (c_.is_sym("*") || c_.is_sym("/")) {
            const bool mul = c_.next().s == "*";
            const double r = unary();
            v = mul ? v * r : v / r;
        }
        return v;
    }
    double unary() {
        Depth guard(this);
        if (c_.is_sym("-")) {
            c_.next();
            return -unary();
        }
        if (c_.is_sym("+")) {
            c_.next();
            return unary();
        }
        return power();
    }
    double power() {
        const double b = atom();
        if (c_.is_sym("^")) {
            c_.next();
            return std::pow(b, unary());
        }
        return b;
    }
    double atom() {
        const Tok &k = c_.peek();
        if (k.kind == Tok::NUM) {
            c_.next();
            return k.v;
        }
        if (k.kind == Tok::SYM && k.s == "(") {
            c_.next();
            const double v = sum();
            c_.expect_sym(")");
            return v;
        }
        if (k.kind == Tok::ID) {
            const std::string name = k.s;
            const int line = k.line;
            c_.next();
            if (name == "pi") return M_PI;
            auto it = env_.find(name);
            if (it != env_.end()) return it->second;
            static const char *fn[] = {"sin", "cos", "tan", "exp", "ln", "sqrt"};
            for (int f = 0; f < 6; ++f)
                if (name == fn[f]) {
                    c_.expect_sym("(");
                    const double a = sum();
                    c_.expect_sym(")");
                    switch (f) {
                        case 0: return std::sin(a);
                        case 1: return std::cos(a);
                        case 2: return std::tan(a);
                        case 3: return std::exp(a);
                        case 4: return std::log(a);
                        default: return std::sqrt(a);
                    }
                }
            bad(line, "unknown name '" + name + "' in an expression");
        }
        bad(k.line, "expected an expression" + c_.got());
    }
};

// the library's gates under their OpenQASM names (primitives U and CX, the
// standard-library names and their common aliases)
struct Builtin {
    uint16_t kind;
    int nq, np;
};
const std::map<std::string, Builtin> &builtins() {
    static const std::map<std::string, Builtin> m = {
        {"U", {QS_U3, 1, 3}},      {"CX", {QS_CX, 2, 0}},     {"id", {QS_I, 1, 0}},     {"u0", {QS_I, 1, 1}},
        {"x", {QS_X, 1, 0}},       {"y", {QS_Y, 1, 0}},       {"z", {QS_Z, 1, 0}},      {"h", {QS_H, 1, 0}},
        {"s", {QS_S, 1, 0}},       {"sdg", {QS_SDG, 1, 0}},   {"t", {QS_T, 1, 0}},      {"tdg", {QS_TDG, 1, 0}},
        {"sx", {QS_SX, 1, 0}},     {"rx", {QS_RX, 1, 1}},     {"ry", {QS_RY, 1, 1}},    {"rz", {QS_RZ, 1, 1}},
        {"u1", {QS_P, 1, 1}},      {"p", {QS_P, 1, 1}},       {"u2", {QS_U2, 1, 2}},    {"u3", {QS_U3, 1, 3}},
        {"u", {QS_U3, 1, 3}},      {"cx", {QS_CX, 2, 0}},     {"cnot", {QS_CX, 2, 0}},  {"cy", {QS_CY, 2, 0}},
        {"cz", {QS_CZ, 2, 0}},     {"ch", {QS_CH, 2, 0}},     {"swap", {QS_SWAP, 2, 0}}, {"iswap", {QS_ISWAP, 2, 0}},
        {"crx", {QS_CRX, 2, 1}},   {"cry", {QS_CRY, 2, 1}},   {"crz", {QS_CRZ, 2, 1}},  {"cu1", {QS_CP, 2, 1}},
        {"cp", {QS_CP, 2, 1}},     {"cphase", {QS_CP, 2, 1}}, {"rzz", {QS_RZZ, 2, 1}},  {"rxx", {QS_RXX, 2, 1}},
        {"ryy", {QS_RYY, 2, 1}},   {"ccx", {QS_CCX, 3, 0}},   {"toffoli", {QS_CCX, 3, 0}},
        {"cswap", {QS_CSWAP, 3, 0}}, {"fredkin", {QS_CSWAP, 3, 0}},
    };
    return m;
}

struct GateDef {
    int index = 0;   // definition order: a body may call only gates defined before it
    std::vector<std::string> params, args;
    size_t body_begin = 0, body_end = 0;   // tokens between the braces
};

constexpr int kMaxQubitsQasm = 63;
constexpr int kMaxInlineDepth = 64;
constexpr long long kMaxCalls = 1ll << 25;   // gate applications, inlined ones included

class Program {
  public:
    Program(const std::vector<Tok> &t, std::vector<qs_gate> &out) : t_(t), out_(out) {}

    int run() {
        Cursor c{&t_, 0, t_.size() - 1};
        while (!c.at_end()) statement(c);
        if (nq_ == 0) bad(t_.back().line, "no qreg declared");
        return nq_;
    }

  private:
    const std::vector<Tok> &t_;
    std::vector<qs_gate> &out_;
    std::map<std::string, std::pair<int, int>> qregs_;   // name -> (first qubit, size)
    std::map<std::string, int> cregs_;
    std::map<std::string, GateDef> defs_;
    std::set<std::string> opaque_;
    int nq_ = 0;
    bool measured_ = false;
    long long calls_ = 0;

    bool declared(const std::string &name) const {
        return qregs_.count(name) || cregs_.count(name) || defs_.count(name) || opaque_.count(name);
    }

    void statement(Cursor &c) {
        const Tok &k = c.peek();
        const int line = k.line;
        if (k.kind != Tok::ID) bad(line, "expected a statement" + c.got());
        const std::string w = k.s;
        if (w == "OPENQASM") {
            c.next();
            const Tok &v = c.next();
            if (v.kind != Tok::NUM || v.v != 2.0) bad(line, "only OpenQASM 2.0 is supported", QS_ERR_UNSUPPORTED);
            c.expect_sym(";");
        } else if (w == "include") {
            c.next();
            const Tok &f = c.next();
            if (f.kind != Tok::STR) bad(line, "expected a file name");
            // the standard library's gates are built in; no other file is read
            if (f.s != "qelib1.inc") bad(line, "include \"" + f.s + "\": only qelib1.inc is known", QS_ERR_UNSUPPORTED);
            c.expect_sym(";");
        } else if (w == "qreg" || w == "creg") {
            c.next();
            const std::string name = c.expect_id("a register name");
            c.expect_sym("[");
            const long size = c.expect_int("a register size");
            c.expect_sym("]");
            c.expect_sym(";");
            if (declared(name)) bad(line, "'" + name + "' is declared twice");
            if (size < 1) bad(line, "register size must be positive");
            if (w == "qreg") {
                if (size > kMaxQubitsQasm - nq_) bad(line, "more than 63 qubits", QS_ERR_UNSUPPORTED);
                qregs_[name] = {nq_, (int)size};
                nq_ += (int)size;
            } else {
                if (size > (1 << 20)) bad(line, "creg larger than 2^20 bits", QS_ERR_UNSUPPORTED);
                cregs_[name] = (int)size;
            }
        } else if (w == "gate") {
            c.next();
            define(c, line);
        } else if (w == "opaque") {
            c.next();
            const std::string name = c.expect_id("a gate name");
            while (!c.at_end() && !c.is_sym(";")) c.next();
            c.expect_sym(";");
            if (declared(name)) bad(line, "'" + name + "' is declared twice");
            opaque_.insert(name);
        } else if (w == "barrier") {
            while (!c.at_end() && !c.is_sym(";")) c.next();
            c.expect_sym(";");
        } else if (w == "measure") {
            c.next();
            const std::vector<int> q = qubit_arg(c);
            c.expect_sym("->");
            const std::string cr = c.expect_id("a classical register");
            if (!cregs_.count(cr)) bad(line, "'" + cr + "' is not a creg");
            if (c.is_sym("[")) {
                c.next();
                const long i = c.expect_int("an index");
                c.expect_sym("]");
                if (i < 0 || i >= cregs_[cr]) bad(line, "index out of range");
                if (q.size() != 1) bad(line, "a register measured into one bit");
            } else if ((int)q.size() != cregs_[cr]) {
                bad(line, "register sizes differ");
            }
            c.expect_sym(";");
            measured_ = true;
        } else if (w == "reset" || w == "if") {
            bad(line, "'" + w + "' is not unitary", QS_ERR_UNSUPPORTED);
        } else {
            call(c);
        }
    }

    void define(Cursor &c, int line) {
        const std::string name = c.expect_id("a gate name");
        if (name == "U" || name == "CX") bad(line, "the primitive " + name + " cannot be redefined");
        if (defs_.count(name) || qregs_.count(name) || cregs_.count(name) || opaque_.count(name))
            bad(line, "'" + name + "' is declared twice");
        GateDef d;
        d.index = (int)defs_.size();
        std::set<std::string> seen;
        if (c.is_sym("(")) {
            c.next();
            while (!c.is_sym(")")) {
                d.params.push_back(c.expect_id("a parameter name"));
                if (!seen.insert(d.params.back()).second) bad(line, "repeated name in the gate's signature");
                if (!c.is_sym(")")) c.expect_sym(",");
            }
            c.next();
        }
        do {
            if (!d.args.empty()) c.expect_sym(",");
            d.args.push_back(c.expect_id("a qubit argument"));
            if (!seen.insert(d.args.back()).second) bad(line, "repeated name in the gate's signature");
        } while (c.is_sym(","));
        c.expect_sym("{");
        d.body_begin = c.pos;
        while (!c.at_end() && !c.is_sym("}")) {
            if (c.is_sym("{")) bad(c.peek().line, "nested braces in a gate body");
            c.next();
        }
        d.body_end = c.pos;
        c.expect_sym("}");
        defs_[name] = d;
    }

    // a top-level qubit argument: a register (all its qubits) or r[i]
    std::vector<int> qubit_arg(Cursor &c) {
        const int line = c.peek().line;
        const std::string r = c.expect_id("a qubit argument");
        auto it = qregs_.find(r);
        if (it == qregs_.end()) bad(line, "'" + r + "' is not a qreg");
        std::vector<int> q;
        if (c.is_sym("[")) {
            c.next();
            const long i = c.expect_int("an index");
            c.expect_sym("]");
            if (i < 0 || i >= it->second.second) bad(line, "index " + std::to_string(i) + " outside " + r);
            q.push_back(it->second.first + (int)i);
        } else {
            for (int i = 0; i < it->second.second; ++i) q.push_back(it->second.first + i);
        }
        return q;
    }

    std::vector<double> param_list(Cursor &c, const std::map<std::string, double> &env) {
        std::vector<double> v;
        if (!c.is_sym("(")) return v;
        c.next();
        while (!c.is_sym(")")) {
            v.push_back(Expr(c, env).sum());
            if (!c.is_sym(")")) c.expect_sym(",");
        }
        c.next();
        return v;
    }

    // a top-level gate call, applied once per index of its register arguments
    void call(Cursor &c) {
        const int line = c.peek().line;
        const std::string name = c.expect_id("a gate name");
        static const std::map<std::string, double> none;
        const std::vector<double> prm = param_list(c, none);
        std::vector<std::vector<int>> args;
        do {
            if (!args.empty()) c.expect_sym(",");
            args.push_back(qubit_arg(c));
        } while (c.is_sym(","));
        c.expect_sym(";");
        size_t k = 1;
        for (auto &a : args)
            if (a.size() > 1) {
                if (k > 1 && a.size() != k) bad(line, "register arguments of different sizes");
                k = a.size();
            }
        for (size_t i = 0; i < k; ++i) {
            std::vector<int> q;
            for (auto &a : args) q.push_back(a.size() > 1 ? a[i] : a[0]);
            apply(name, prm, q, line, 0, -1);
        }
    }

    // `limit`: inside a body, only gates defined before index `limit` (-1: any)
    void apply(const std::string &name, const std::vector<double> &prm, const std::vector<int> &q, int line,
               int depth, int limit) {
        if (depth > kMaxInlineDepth) bad(line, "gate definitions nested too deeply", QS_ERR_UNSUPPORTED);
        if (++calls_ > kMaxCalls) bad(line, "more than 2^25 gate applications", QS_ERR_UNSUPPORTED);
        for (size_t i = 0; i < q.size(); ++i)
            for (size_t j = i + 1; j < q.size(); ++j)
                if (q[i] == q[j]) bad(line, "gate '" + name + "' repeats a qubit");
        auto d = defs_.find(name);
        if (d != defs_.end() && (limit < 0 || d->second.index < limit)) {
            expand(name, d->second, prm, q, line, depth);
            return;
        }
        auto b = builtins().find(name);
        if (b == builtins().end() && name == "cu3" && d == defs_.end()) {
            cu3(prm, q, line);
            return;
        }
        if (b == builtins().end() && name == "sxdg" && d == defs_.end()) {   // SX^4 = X^2 = I: SX^-1 = SX^3
            if (q.size() != 1) bad(line, "gate 'sxdg' takes 1 qubit(s)");
            if (!prm.empty()) bad(line, "gate 'sxdg' takes 0 parameter(s)");
            for (int r = 0; r < 3; ++r) emit("sxdg", QS_SX, {}, {q[0]}, line);
            return;
        }
        if (b == builtins().end() && (name == "c3x" || name == "c4x") && d == defs_.end()) {
            const int k = name == "c3x" ? 3 : 4;
            if ((int)q.size() != k + 1) bad(line, "gate '" + name + "' takes " + std::to_string(k + 1) + " qubit(s)");
            if (!prm.empty()) bad(line, "gate '" + name + "' takes 0 parameter(s)");
            mcx(q, line);
            return;
        }
        if (b == builtins().end()) {
            if (d != defs_.end()) bad(line, "gate '" + name + "' is used before its definition");
            if (opaque_.count(name)) bad(line, "opaque gate '" + name + "'", QS_ERR_UNSUPPORTED);
            bad(line, "gate '" + name + "' is not in the library's gate set and has no definition",
                QS_ERR_UNSUPPORTED);
        }
        const Builtin &g = b->second;
        if ((int)q.size() != g.nq)
            bad(line, "gate '" + name + "' takes " + std::to_string(g.nq) + " qubit(s)");
        if ((int)prm.size() != g.np)
            bad(line, "gate '" + name + "' takes " + std::to_string(g.np) + " parameter(s)");
        emit(name, g.kind, prm, q, line);
    }

    void emit(const std::string &name, uint16_t kind, const std::vector<double> &prm, const std::vector<int> &q,
              int line) {
        if (measured_) bad(line, "a unitary gate after a measurement", QS_ERR_UNSUPPORTED);
        for (double v : prm)
            if (!std::isfinite(v)) bad(line, "gate '" + name + "': angle is not finite");
        qs_gate r;
        std::memset(&r, 0, sizeof r);
        r.kind = kind;
        r.nw = (uint8_t)q.size();
        for (size_t i = 0; i < q.size(); ++i) r.w[i] = q[i];
        if (kind != QS_I)
            for (size_t i = 0; i < prm.size() && i < 3; ++i) r.p[i] = prm[i];
        r.param_idx = -1;
        r.dense = nullptr;
        out_.push_back(r);
    }

    // X on the last of q controlled by all the others (m = |q| qubits), with no
    // ancilla: H on the target turns it into the phase pi x_1 ... x_m, and
    // x_1 ... x_m = 2^(1-m) sum over nonempty subsets S of (-1)^(|S|+1)
    // (parity of x over S) (inclusion-exclusion over parities).  Each
    // parity is gathered onto the highest qubit of S by CX from the others,
    // takes P(+-pi / 2^(m-1)), and the CX are undone.
    void mcx(const std::vector<int> &q, int line) {
        const int m = (int)q.size(), t = q[m - 1];
        emit("mcx", QS_H, {}, {t}, line);
        for (unsigned S = 1; S < (1u << m); ++S) {
            int top = -1, size = 0;
            for (int i = 0; i < m; ++i)
                if ((S >> i) & 1) {
                    top = i;
                    ++size;
                }
            const double ang = ((size & 1) ? 1.0 : -1.0) * M_PI / (double)(1u << (m - 1));
            for (int i = 0; i < top; ++i)
                if ((S >> i) & 1) emit("mcx", QS_CX, {}, {q[i], q[top]}, line);
            emit("mcx", QS_P, {ang}, {q[top]}, line);
            for (int i = top - 1; i >= 0; --i)
                if ((S >> i) & 1) emit("mcx", QS_CX, {}, {q[i], q[top]}, line);
        }
        emit("mcx", QS_H, {}, {t}, line);
    }

    // cu3(theta, phi, lambda) c, t: controlled-U3, U3 = e^{i(phi+lambda)/2} RZ(phi) RY(theta) RZ(lambda).
    // With A = RZ(phi) RY(theta/2), B = RY(-theta/2) RZ(-(phi+lambda)/2) and
    // C = RZ((lambda-phi)/2): A B C = I and A X B X C = e^{-i(phi+lambda)/2} U3, so
    // controlled-U3 = P((phi+lambda)/2) on c after C, CX, B, CX, A on t (the
    // two-CX construction of a controlled single-qubit gate), exactly.
    void cu3(const std::vector<double> &prm, const std::vector<int> &q, int line) {
        if (q.size() != 2) bad(line, "gate 'cu3' takes 2 qubit(s)");
        if (prm.size() != 3) bad(line, "gate 'cu3' takes 3 parameter(s)");
        const double th = prm[0], ph = prm[1], la = prm[2];
        const int c = q[0], t = q[1];
        emit("cu3", QS_RZ, {(la - ph) / 2}, {t}, line);
        emit("cu3", QS_CX, {}, {c, t}, line);
        emit("cu3", QS_RZ, {-(ph + la) / 2}, {t}, line);
        emit("cu3", QS_RY, {-th / 2}, {t}, line);
        emit("cu3", QS_CX, {}, {c, t}, line);
        emit("cu3", QS_RY, {th / 2}, {t}, line);
        emit("cu3", QS_RZ, {ph}, {t}, line);
        emit("cu3", QS_P, {(ph + la) / 2}, {c}, line);
    }

    void expand(const std::string &name, const GateDef &d, const std::vector<double> &prm,
                const std::vector<int> &q, int line, int depth) {
        if (prm.size() != d.params.size())
            bad(line, "gate '" + name + "' takes " + std::to_string(d.params.size()) + " parameter(s)");
        if (q.size() != d.args.size())
            bad(line, "gate '" + name + "' takes " + std::to_string(d.args.size()) + " qubit(s)");
        std::map<std::string, double> env;
        for (size_t i = 0; i < prm.size(); ++i) env[d.params[i]] = prm[i];
        std::map<std::string, int> qb;
        for (size_t i = 0; i < q.size(); ++i) qb[d.args[i]] = q[i];
        Cursor c{&t_, d.body_begin, d.body_end};
        while (!c.at_end()) {
            const int bl = c.peek().line;
            if (c.is_id("barrier")) {
                while (!c.at_end() && !c.is_sym(";")) c.next();
                c.expect_sym(";");
                continue;
            }
            const std::string callee = c.expect_id("a gate call");
            const std::vector<double> cp = param_list(c, env);
            std::vector<int> cq;
            do {
                if (!cq.empty()) c.expect_sym(",");
                const std::string a = c.expect_id("a qubit argument");
                auto it = qb.find(a);
                if (it == qb.end()) bad(bl, "'" + a + "' is not an argument of gate '" + name + "'");
                cq.push_back(it->second);
            } while (c.is_sym(","));
            c.expect_sym(";");
            apply(callee, cp, cq, bl, depth + 1, d.index);
        }
    }
};

}  // namespace

qs_status parse_qasm(const char *src, std::vector<qs_gate> &out, int &n_qubits, std::string &err) {
    out.clear();
    n_qubits = 0;
    if (!src) {
        err = "source is NULL";
        return QS_ERR_INVALID_ARG;
    }
    try {
        const std::vector<Tok> toks = lex(src);
        Program p(toks, out);
        n_qubits = p.run();
    } catch (const ParseError &e) {
        out.clear();
        n_qubits = 0;
        err = e.msg;
        return e.st;
    }
    return QS_OK;
}

}  // namespace qs
