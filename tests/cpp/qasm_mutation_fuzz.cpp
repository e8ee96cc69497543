// Mutation fuzz of the OpenQASM parser in-process, built with
// AddressSanitizer and UBSan by tests/test_qasm_fuzz.py: a valid program
// (user gates, expressions, broadcast, cu3, barrier, measurement) is mutated
// by erasing, inserting tokens from the grammar's vocabulary, replacing bytes
// and duplicating slices; every program must come back with a status and no
// sanitizer report.  Arguments: seed, iterations.  Prints "ok=<n> err=<n>".
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>
#include "qs_qasm.h"
int main(int argc, char **argv) {
    std::mt19937_64 rng(argc > 1 ? atoi(argv[1]) : 1);
    const std::string base =
        "OPENQASM 2.0;\ninclude \"qelib1.inc\";\nqreg q[5];\nqreg r[3];\ncreg c[5];\n"
        "gate zz(t) a, b { cx a, b; rz(t) b; cx a, b; }\n"
        "gate lay(t, f) a, b { ry(f) a; zz(t*pi/2) a, b; u3(f, -t, 2^-1) b; }\n"
        "h q;\nlay(0.3, sin(0.2)) q[0], r[1];\ncx q[1], r[2];\ncu1(pi/4) q[2], q[3];\ncu3(1,2,3) q[0], r[0];\n"
        "barrier q, r;\nccx q[0], q[1], r[0];\nswap r[0], q[4];\nmeasure q -> c;\n";
    const char *vocab[] = {"OPENQASM", "2.0", "include", "\"qelib1.inc\"", "qreg", "creg", "gate", "opaque", "barrier",
                           "measure", "q", "r", "a", "b", "t", "[", "]", "(", ")", "{", "}", ";", ",", "->", "+", "-",
                           "*", "/", "^", "pi", "sin", "sqrt", "0", "1", "7", "1e308", "99999999999999999999",
                           "h", "cx", "u3", "cu3", "c3x", "c4x", "zz", "lay", "U", "CX", "//", "/*", "*/", "\"", "\n", "((((", "----"};
    long ok = 0, err = 0;
    const int iters = argc > 2 ? atoi(argv[2]) : 20000;
    for (int it = 0; it < iters; ++it) {
        std::string s = base;
        int muts = 1 + rng() % 4;
        for (int m = 0; m < muts; ++m) {
            size_t pos = rng() % (s.size() + 1);
            switch (rng() % 4) {
                case 0: if (!s.empty()) s.erase(pos < s.size() ? pos : s.size() - 1, 1 + rng() % 6); break;
                case 1: s.insert(pos, std::string(" ") + vocab[rng() % (sizeof vocab / sizeof *vocab)] + " "); break;
                case 2: if (pos < s.size()) s[pos] = (char)(1 + rng() % 126); break;
                default: s.insert(pos, s.substr(rng() % s.size(), rng() % 40)); break;
            }
        }
        std::vector<qs_gate> g; int n; std::string e;
        if (qs::parse_qasm(s.c_str(), g, n, e) == QS_OK) ++ok; else ++err;
    }
    std::printf("ok=%ld err=%ld\n", ok, err);
}
