// Build-time tool: compiles amplitude-model JSON files and writes the
// header of compile-time model structures the per-event kernels are
// specialised on.  Usage: shapegen OUT.h MODEL.json [MODEL.json ...]
#include <fstream>
#include <iostream>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "model.hpp"

using namespace tdmix;

static std::string fn(const char* name, const std::vector<int>& v) {
  std::ostringstream s;
  s << "  __host__ __device__ static constexpr int " << name << "(int i) {\n    switch (i) {\n";
  for (size_t k = 0; k < v.size(); ++k) s << "      case " << k << ": return " << v[k] << ";\n";
  s << "      default: return -1;\n    }\n  }\n";
  return s.str();
}

int main(int argc, char** argv) {
  if (argc < 2) {
    std::cerr << "usage: shapegen OUT.h MODEL.json...\n";
    return 2;
  }
  std::ostringstream out;
  out << "// Generated by shapegen from the amplitude-model files; do not edit.\n#pragma once\n"
      << "namespace tdmix {\nnamespace shapes {\n";
  std::set<std::string> seen;
  std::vector<std::string> names;
  for (int a = 2; a < argc; ++a) {
    std::ifstream f(argv[a]);
    std::stringstream buf;
    buf << f.rdbuf();
    CompiledModel m;
    try {
      m = compile_model(buf.str());
    } catch (const std::exception& e) {
      std::cerr << argv[a] << ": " << e.what() << "\n";
      return 1;
    }
    std::string sig = m.signature();
    if (!seen.insert(sig).second) continue;
    std::string nm = "Shape" + std::to_string(names.size());
    names.push_back(nm);
    std::vector<int> tb0, tb1, bres, bs, bx;
    for (const Term& t : m.terms) {
      tb0.push_back(t.b[0]);
      tb1.push_back(t.b[1]);
    }
    for (const BWInstance& b : m.bws) {
      bres.push_back(b.res);
      bs.push_back(b.splane);
      bx.push_back(b.xplane);
    }
    out << "// " << (m.name.empty() ? argv[a] : m.name) << "\nstruct " << nm << " {\n"
        << "  static constexpr int U = " << m.U << ", NO = " << m.NO << ", NB = " << m.NB() << ", NR = " << m.NR()
        << ", NS = " << m.NS() << ", NX = " << m.NX() << ";\n"
        << fn("tb0", tb0) << fn("tb1", tb1) << fn("bres", bres) << fn("bs", bs) << fn("bx", bx)
        << "  static const char* sig() { return \"" << sig << "\"; }\n};\n";
  }
  out << "}  // namespace shapes\n}  // namespace tdmix\n#define TDMIX_FOR_EACH_SHAPE(X)";
  for (auto& n : names) out << " X(" << n << ")";
  out << "\n";
  std::ofstream o(argv[1]);
  o << out.str();
  return o ? 0 : 1;
}
