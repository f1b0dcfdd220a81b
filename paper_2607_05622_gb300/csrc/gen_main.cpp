// Build-time generator of the class-specialised integral code.
//
// Writes one header with, for every class that gen_class() selects, the
// straight-line vertical and horizontal recurrences of codegen.cpp (templates
// over the arithmetic type) and a GenClass<la,lb,lc,ld> specialisation that
// gives the class's sizes as compile-time constants; plus the X-macro
// LTJK_GEN_CLASSES(X) listing the classes, from which the library builds its
// kernel dispatch.  Run by the library build before nvcc, on the build host.
// Usage: gen_main <out.inc>
#include <cstdio>
#include <fstream>
#include <string>

#include "ltjk_internal.h"

using namespace ltjk;

int main(int argc, char **argv) {
  if (argc != 2) {
    std::fprintf(stderr, "usage: gen_main <out.inc>\n");
    return 2;
  }
  ProgramSet ps;
  try {
    build_programs(ps);
  } catch (const std::exception &e) {
    std::fprintf(stderr, "gen_main: %s\n", e.what());
    return 1;
  }
  std::string body, spec, list;
  for (int la = 0; la <= kMaxL; ++la)
    for (int lb = 0; lb <= la; ++lb)
      for (int lc = 0; lc <= kMaxL; ++lc)
        for (int ld = 0; ld <= lc; ++ld) {
          if (!gen_class(la, lb, lc, ld)) continue;
          const ClassProg &p = ps.progs[quartet_index(la, lb, lc, ld, 0)];
          const std::string cls = std::to_string(la) + std::to_string(lb) + std::to_string(lc) +
                                  std::to_string(ld);
          const std::string name = "gen_c" + cls;
          try {
            body += emit_class_source(ps, la, lb, lc, ld, 0, name) + "\n";
          } catch (const std::exception &e) {
            std::fprintf(stderr, "gen_main: class %s: %s\n", cls.c_str(), e.what());
            return 1;
          }
          spec += "template <> struct GenClass<" + std::to_string(la) + ", " + std::to_string(lb) + ", " +
                  std::to_string(lc) + ", " + std::to_string(ld) + "> {\n" +
                  "  static constexpr int kLtot = " + std::to_string(p.ltot) + ";\n" +
                  "  static constexpr int kAcc = " + std::to_string(p.acc_total) + ";\n" +
                  "  static constexpr int kOut = " + std::to_string(p.nout) + ";\n" +
                  "  static constexpr int kNh = " + std::to_string(p.nh) + ";\n" +
                  "  template <typename Real, int AS = 1>\n  static LTJK_GEN_FN void vrr(const Real *b, const Real *cf, "
                  "const Real *h, Real *acc) {\n    " + name + "_vrr<Real, AS>(b, cf, h, acc);\n  }\n" +
                  "  template <typename Real, int AS = 1, int OS = 1>\n  static LTJK_GEN_FN void hrr(const Real *acc, "
                  "const Real *X, Real *out) {\n    " + name + "_hrr<Real, AS, OS>(acc, X, out);\n  }\n};\n";
          list += " X(" + std::to_string(la) + ", " + std::to_string(lb) + ", " + std::to_string(lc) + ", " +
                  std::to_string(ld) + ")";
        }
  std::ofstream f(argv[1]);
  f << "// Generated by csrc/gen_main.cpp at build time; do not edit.\n#pragma once\n\n";
  f << "#ifndef LTJK_GEN_FN\n#error \"define LTJK_GEN_FN before including the generated classes\"\n#endif\n\n";
  f << "namespace ltjk {\n\n" << body;
  f << "template <int LA, int LB, int LC, int LD>\nstruct GenClass;\n\n" << spec << "\n";
  f << "}  // namespace ltjk\n\n#define LTJK_GEN_CLASSES(X)" << list << "\n";
  return f ? 0 : 1;
}
