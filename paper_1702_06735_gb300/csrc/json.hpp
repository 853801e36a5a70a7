// Minimal JSON reader for model descriptions (objects, arrays, strings,
// numbers, true/false/null).  Host code only.
#pragma once
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

namespace tdmix {

struct Json {
  enum Kind { Null, Bool, Number, String, Array, Object } kind = Null;
  bool b = false;
  double num = 0.0;
  std::string str;
  std::vector<Json> arr;
  std::vector<std::pair<std::string, Json>> obj;

  const Json* find(const std::string& key) const {
    for (auto& kv : obj)
      if (kv.first == key) return &kv.second;
    return nullptr;
  }
  const Json& at(const std::string& key) const {
    const Json* j = find(key);
    if (!j) throw std::runtime_error("model JSON: missing key '" + key + "'");
    return *j;
  }
  double number() const {
    if (kind != Number) throw std::runtime_error("model JSON: expected a number");
    return num;
  }
  const std::string& string() const {
    if (kind != String) throw std::runtime_error("model JSON: expected a string");
    return str;
  }
  bool boolean() const {
    if (kind != Bool) throw std::runtime_error("model JSON: expected true/false");
    return b;
  }
  const std::vector<Json>& array() const {
    if (kind != Array) throw std::runtime_error("model JSON: expected an array");
    return arr;
  }
};

Json parse_json(const std::string& text);

}  // namespace tdmix
