#include "model.hpp"

#include <algorithm>
#include <cmath>
#include <sstream>
#include <stdexcept>

#include "json.hpp"

namespace tdmix {
namespace {

int spin_of(const std::string& s) {
  if (s == "VV_S") return SPIN_VV_S;
  if (s == "VV_P") return SPIN_VV_P;
  if (s == "VV_D") return SPIN_VV_D;
  if (s == "AP_S") return SPIN_AP_S;
  if (s == "NR") return SPIN_NR;
  throw std::runtime_error("model: unknown spin factor '" + s + "'");
}

int shape_of(const std::string& s) {
  if (s == "MDW") return SHAPE_MDW;
  if (s == "CONST") return SHAPE_CONST;
  if (s == "NR") return SHAPE_NONE;
  throw std::runtime_error("model: unknown lineshape '" + s + "'");
}

bool get_bool(const Json& o, const char* key, bool dflt) {
  const Json* j = o.find(key);
  return j ? j->boolean() : dflt;
}

}  // namespace

CompiledModel compile_model(const std::string& text) {
  Json d = parse_json(text);
  CompiledModel m;
  if (const Json* n = d.find("name")) m.name = n->string();
  m.parent_mass = d.at("parent_mass").number();
  const auto& fs = d.at("final_state").array();
  if (fs.size() != 4) throw std::runtime_error("model: final_state must list four particles");
  for (int i = 0; i < 4; ++i) m.masses[i] = fs[i].at("mass").number();
  m.tau = d.at("tau").number();
  if (!(m.tau > 0)) throw std::runtime_error("model: tau must be positive");
  m.r_res = d.at("r_resonance").number();
  m.r_parent = d.at("r_parent").number();
  if (const Json* b = d.find("bose_swap"); b && b->kind != Json::Null) {
    const auto& a = b->array();
    if (a.size() != 2) throw std::runtime_error("model: bose_swap needs two indices");
    m.bose[0] = int(a[0].number());
    m.bose[1] = int(a[1].number());
    if (m.bose[0] < 0 || m.bose[0] > 3 || m.bose[1] < 0 || m.bose[1] > 3 || m.bose[0] == m.bose[1] ||
        m.masses[m.bose[0]] != m.masses[m.bose[1]])
      throw std::runtime_error("model: bose_swap must name two distinct identical particles");
  }
  m.x = d.at("x").number();
  m.y = d.at("y").number();
  m.float_xy = get_bool(d, "float_xy", true);
  m.dedup = get_bool(d, "dedup", true);
  if (const Json* r = d.find("time_resolution"); r && r->kind != Json::Null) {
    m.sigma_t = r->number();
    if (!(m.sigma_t >= 0) || !std::isfinite(m.sigma_t))
      throw std::runtime_error("model: time_resolution must be a width >= 0 (ps)");
  }
  if (const Json* bg = d.find("background"); bg && bg->kind != Json::Null) {
    m.bkg_fraction = bg->at("fraction").number();
    m.bkg_tau = bg->at("tau").number();
    if (!(m.bkg_fraction >= 0 && m.bkg_fraction < 1) || !(m.bkg_tau > 0) || !std::isfinite(m.bkg_tau))
      throw std::runtime_error("model: background needs 0 <= fraction < 1 and tau > 0 (ps)");
  }

  for (const Json& r : d.at("resonances").array()) {
    ResonanceDef rd;
    rd.name = r.at("name").string();
    rd.mass = r.at("mass").number();
    rd.width = r.at("width").number();
    rd.shape = shape_of(r.at("shape").string());
    if (const Json* L = r.find("L")) rd.L = int(L->number());
    if (rd.shape == SHAPE_MDW) {
      const auto& dm = r.at("daughter_masses").array();
      if (dm.size() != 2) throw std::runtime_error("model: daughter_masses needs two entries");
      rd.ma = dm[0].number();
      rd.mb = dm[1].number();
      if (rd.L < 0 || rd.L > 2) throw std::runtime_error("model: L must be 0, 1 or 2");
    }
    rd.floating = get_bool(r, "float", true);
    for (auto& o : m.res)
      if (o.name == rd.name) throw std::runtime_error("model: duplicate resonance '" + rd.name + "'");
    m.res.push_back(rd);
  }
  if (m.res.size() > size_t(kMaxRes)) throw std::runtime_error("model: too many resonances");

  for (const Json& c : d.at("chains").array()) {
    ChainDef cd;
    if (const Json* n = c.find("name")) cd.name = n->string();
    const std::string& amp = c.at("amp").string();
    if (amp == "A") cd.amp = 0;
    else if (amp == "Abar") cd.amp = 1;
    else throw std::runtime_error("model: amp must be 'A' or 'Abar'");
    cd.spin = spin_of(c.at("spin").string());
    if (const Json* rl = c.find("resonances")) {
      for (const Json& rn : rl->array()) {
        int k = -1;
        for (size_t i = 0; i < m.res.size(); ++i)
          if (m.res[i].name == rn.string()) k = int(i);
        if (k < 0) throw std::runtime_error("model: chain names unknown resonance '" + rn.string() + "'");
        cd.res.push_back(k);
      }
    }
    size_t need = cd.spin == SPIN_NR ? 0 : 2;
    if (cd.res.size() != need)
      throw std::runtime_error("model: chain '" + cd.name + "' needs " + std::to_string(need) + " resonances");
    if (const Json* p = c.find("particles")) {
      const auto& a = p->array();
      if (a.size() != 4) throw std::runtime_error("model: particles needs four indices");
      int seen = 0;
      for (int i = 0; i < 4; ++i) {
        cd.parts[i] = int(a[i].number());
        if (cd.parts[i] < 0 || cd.parts[i] > 3) throw std::runtime_error("model: particle index out of range");
        seen |= 1 << cd.parts[i];
      }
      if (seen != 15) throw std::runtime_error("model: particles must be a permutation of 0..3");
    }
    const auto& co = c.at("coef").array();
    if (co.size() != 2) throw std::runtime_error("model: coef needs [re, im]");
    cd.cre = co[0].number();
    cd.cim = co[1].number();
    cd.floating = get_bool(c, "float", true);
    m.chains.push_back(cd);
  }
  if (m.chains.empty()) throw std::runtime_error("model: no chains");
  if (m.chains.size() > size_t(kMaxChains)) throw std::runtime_error("model: too many chains");

  // components
  m.NO = m.bose[0] >= 0 ? 2 : 1;
  std::vector<int> comp_rep;  // representative chain of each component
  for (size_t i = 0; i < m.chains.size(); ++i) {
    const ChainDef& c = m.chains[i];
    int found = -1;
    if (m.dedup) {
      for (size_t j = 0; j < comp_rep.size(); ++j) {
        const ChainDef& r = m.chains[comp_rep[j]];
        if (r.spin == c.spin && r.res == c.res && std::equal(r.parts, r.parts + 4, c.parts)) found = int(j);
      }
    }
    if (found < 0) {
      found = int(comp_rep.size());
      comp_rep.push_back(int(i));
    }
    m.chain_comp.push_back(found);
  }
  m.U = int(comp_rep.size());
  if (m.U > kMaxComp) throw std::runtime_error("model: too many distinct components");
  for (size_t i = 0; i < m.chains.size(); ++i)
    for (size_t k = 0; k < i; ++k)
      if (m.chain_comp[i] == m.chain_comp[k] && m.chains[i].amp == m.chains[k].amp)
        throw std::runtime_error("model: chains '" + m.chains[k].name + "' and '" + m.chains[i].name +
                                 "' are the same amplitude term");

  auto splane_of = [&](int mask) {
    for (size_t i = 0; i < m.splane_mask.size(); ++i)
      if (m.splane_mask[i] == mask) return int(i);
    m.splane_mask.push_back(mask);
    return int(m.splane_mask.size()) - 1;
  };
  auto xplane_of = [&](int sp, const ResonanceDef& r) {
    for (size_t i = 0; i < m.xplanes.size(); ++i) {
      const XPlane& x = m.xplanes[i];
      if (x.splane == sp && x.ma == r.ma && x.mb == r.mb && x.L == r.L) return int(i);
    }
    m.xplanes.push_back({sp, r.ma, r.mb, r.L});
    return int(m.xplanes.size()) - 1;
  };
  auto bw_of = [&](int res, int mask) {
    if (m.res[res].shape == SHAPE_NONE) return -1;
    int sp = splane_of(mask);
    for (size_t i = 0; i < m.bws.size(); ++i)
      if (m.bws[i].res == res && m.bws[i].splane == sp) return int(i);
    int xp = m.res[res].shape == SHAPE_MDW ? xplane_of(sp, m.res[res]) : -1;
    m.bws.push_back({res, sp, xp});
    return int(m.bws.size()) - 1;
  };

  for (int j = 0; j < m.U; ++j) {
    const ChainDef& c = m.chains[comp_rep[j]];
    for (int o = 0; o < m.NO; ++o) {
      Term t;
      t.spin = c.spin;
      for (int k = 0; k < 4; ++k) {
        int p = c.parts[k];
        if (o == 1) p = p == m.bose[0] ? m.bose[1] : (p == m.bose[1] ? m.bose[0] : p);
        t.parts[k] = p;
      }
      t.b[0] = t.b[1] = -1;
      int a = 1 << t.parts[0], b = 1 << t.parts[1], cc = 1 << t.parts[2], dd = 1 << t.parts[3];
      if (c.spin == SPIN_VV_S || c.spin == SPIN_VV_P || c.spin == SPIN_VV_D) {
        t.b[0] = bw_of(c.res[0], a | b);
        t.b[1] = bw_of(c.res[1], cc | dd);
      } else if (c.spin == SPIN_AP_S) {
        t.b[0] = bw_of(c.res[0], a | b | cc);
        t.b[1] = bw_of(c.res[1], a | b);
      }
      m.terms.push_back(t);
    }
  }
  if (m.NB() > kMaxBW || m.NS() > kMaxSPlanes || m.NX() > kMaxXPlanes)
    throw std::runtime_error("model: too many distinct lineshapes or invariants");
  return m;
}

std::string CompiledModel::signature() const {
  std::ostringstream s;
  s << "U" << U << "O" << NO << "B" << NB() << "R" << NR() << "S" << NS() << "X" << NX() << ":T";
  for (const Term& t : terms) s << t.b[0] << "," << t.b[1] << ";";
  s << ":B";
  for (const BWInstance& b : bws) s << b.res << "," << b.splane << "," << b.xplane << ";";
  return s.str();
}

std::vector<double> CompiledModel::default_params() const {
  std::vector<double> p;
  for (const ChainDef& c : chains) {
    p.push_back(c.cre);
    p.push_back(c.cim);
  }
  for (const ResonanceDef& r : res) {
    p.push_back(r.mass);
    p.push_back(r.width);
  }
  p.push_back(x);
  p.push_back(y);
  return p;
}

std::vector<int> CompiledModel::floating_mask() const {
  std::vector<int> f;
  for (const ChainDef& c : chains) {
    f.push_back(c.floating);
    f.push_back(c.floating);
  }
  for (const ResonanceDef& r : res) {
    f.push_back(r.floating);
    f.push_back(r.floating);
  }
  f.push_back(float_xy);
  f.push_back(float_xy);
  return f;
}

}  // namespace tdmix
