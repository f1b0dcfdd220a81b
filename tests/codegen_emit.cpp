// Test infrastructure: writes the straight-line source of every class program
// (paper_2607_05622_gb300/csrc/codegen.cpp) to one header, with a dispatch
// table indexed like the program set, for tests/codegen_eval.cpp.
// Usage: codegen_emit <out.h> <deriv 0|1> [largest l]
#include <cstdio>
#include <fstream>
#include <string>

#include "ltjk_internal.h"

using namespace ltjk;

int main(int argc, char **argv) {
  if (argc != 3 && argc != 4) return 2;
  const int deriv = std::stoi(argv[2]);
  const int lmax = argc == 4 ? std::stoi(argv[3]) : kMaxL;
  ProgramSet ps;
  build_programs(ps);
  std::ofstream f(argv[1]);
  f << "// generated by tests/codegen_emit.cpp\n#pragma once\n#include <cmath>\n";
  f << "#ifndef LTJK_HD\n#define LTJK_HD\n#endif\n#define LTJK_GEN_FN LTJK_HD inline\n\n";
  std::string table;
  for (int la = 0; la <= lmax; ++la)
    for (int lb = 0; lb <= la; ++lb)
      for (int lc = 0; lc <= lmax; ++lc)
        for (int ld = 0; ld <= lc; ++ld) {
          const std::string name = "c" + std::to_string(la) + std::to_string(lb) + std::to_string(lc) +
                                   std::to_string(ld) + "d" + std::to_string(deriv);
          f << emit_class_source(ps, la, lb, lc, ld, deriv, name) << "\n";
          table += "  {" + std::to_string(la) + ", " + std::to_string(lb) + ", " + std::to_string(lc) +
                   ", " + std::to_string(ld) + ", &" + name + "_vrr<double>, &" + name + "_hrr<double>},\n";
        }
  f << "struct GenClass {\n  int la, lb, lc, ld;\n"
    << "  void (*vrr)(const double *, const double *, const double *, double *);\n"
    << "  void (*hrr)(const double *, const double *, double *);\n};\n";
  f << "static const GenClass kGenClasses[] = {\n" << table << "};\n";
  return f ? 0 : 1;
}
