// OpenQASM 2.0 import: the unitary subset of a program as gate records
// (Sec. 3.3 "OpenQASM Integration": standard gate set, parameterised
// rotations, user-defined gates inlined with nested definitions,
// register-wide operations; App. B.1: names normalised into the detector's
// vocabulary, barriers skipped).
#pragma once

#include <string>
#include <vector>

#include "qs.h"

namespace qs {

// Parses `src` (NUL-terminated).  On success fills `out` (param_idx = -1,
// dense = NULL), `n_qubits` (the sum of all qreg sizes) and returns QS_OK;
// otherwise QS_ERR_INVALID_ARG (syntax, undeclared names, arity, repeated
// qubits) or QS_ERR_UNSUPPORTED (a gate outside the library's set that no
// `gate` definition provides, opaque gates, reset, if, a unitary gate after a
// measurement, includes other than qelib1.inc), with `err` = "line L: ...".
qs_status parse_qasm(const char *src, std::vector<qs_gate> &out, int &n_qubits, std::string &err);

}  // namespace qs
