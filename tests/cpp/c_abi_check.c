/* The C ABI from plain C (C11): include qs.h, link libqs.so, and call the
 * entry points that need no GPU: version, OpenQASM import, plan description,
 * argument validation and the error message.  Prints "OK <passes>" or the
 * first failure. */
#include <stdio.h>
#include <string.h>

#include "qs.h"

int main(void) {
    const char *src =
        "OPENQASM 2.0;\n"
        "include \"qelib1.inc\";\n"
        "qreg q[14];\n"
        "h q;\n"
        "cu1(pi/2) q[1], q[0];\n"
        "cx q[0], q[13];\n"
        "rzz(0.25) q[3], q[9];\n";
    qs_gate *gates = NULL;
    size_t n_gates = 0;
    int n = 0;
    if (qs_qasm_parse(src, &gates, &n_gates, &n) != QS_OK) {
        printf("parse: %s\n", qs_last_error());
        return 1;
    }
    if (n != 14 || n_gates != 17 || gates[14].kind != QS_CP || gates[15].kind != QS_CX) {
        printf("records: n=%d gates=%zu\n", n, n_gates);
        return 1;
    }
    char buf[4096];
    int passes = 0;
    qs_opts o;
    memset(&o, 0, sizeof o);
    o.mode = QS_MODE_FUSED;
    if (qs_plan_describe(n, gates, n_gates, &o, buf, sizeof buf, &passes) != QS_OK || passes < 1 ||
        strncmp(buf, "FUSED n=14", 10) != 0) {
        printf("describe: %s\n", qs_last_error());
        return 1;
    }
    gates[0].w[0] = 99; /* out of range: rejected with a message */
    if (qs_plan_describe(n, gates, n_gates, &o, buf, sizeof buf, &passes) != QS_ERR_INVALID_ARG ||
        strlen(qs_last_error()) == 0) {
        printf("validation\n");
        return 1;
    }
    qs_qasm_free(gates);
    if (qs_qasm_parse("qreg q[1]; foo q[0];", &gates, &n_gates, &n) != QS_ERR_UNSUPPORTED || gates != NULL ||
        n_gates != 0 || strstr(qs_last_error(), "line 1") == NULL) {
        printf("error path\n");
        return 1;
    }
    if (strstr(qs_version(), "sm_103a") == NULL) {
        printf("version\n");
        return 1;
    }
    printf("OK %d\n", passes);
    return 0;
}
