#include "json.hpp"

#include <cstdlib>

namespace tdmix {
namespace {

struct Parser {
  const std::string& s;
  size_t i = 0;
  explicit Parser(const std::string& t) : s(t) {}

  [[noreturn]] void fail(const char* what) {
    throw std::runtime_error(std::string("model JSON: ") + what + " at offset " + std::to_string(i));
  }
  void ws() {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\t' || s[i] == '\r')) ++i;
  }
  bool lit(const char* w) {
    size_t n = 0;
    while (w[n]) ++n;
    if (s.compare(i, n, w) == 0) {
      i += n;
      return true;
    }
    return false;
  }
  std::string str() {
    if (s[i] != '"') fail("expected string");
    ++i;
    std::string out;
    while (i < s.size() && s[i] != '"') {
      char c = s[i++];
      if (c == '\\') {
        if (i >= s.size()) fail("bad escape");
        char e = s[i++];
        switch (e) {
          case 'n': out += '\n'; break;
          case 't': out += '\t'; break;
          case 'r': out += '\r'; break;
          case 'b': out += '\b'; break;
          case 'f': out += '\f'; break;
          case 'u': {  // keep ASCII code points, replace others
            if (i + 4 > s.size()) fail("bad \\u escape");
            unsigned v = std::strtoul(s.substr(i, 4).c_str(), nullptr, 16);
            i += 4;
            out += v < 128 ? char(v) : '?';
            break;
          }
          default: out += e;
        }
      } else {
        out += c;
      }
    }
    if (i >= s.size()) fail("unterminated string");
    ++i;
    return out;
  }
  Json value() {
    ws();
    if (i >= s.size()) fail("unexpected end");
    Json j;
    char c = s[i];
    if (c == '{') {
      j.kind = Json::Object;
      ++i;
      ws();
      if (s[i] == '}') { ++i; return j; }
      for (;;) {
        ws();
        std::string k = str();
        ws();
        if (s[i] != ':') fail("expected ':'");
        ++i;
        j.obj.emplace_back(k, value());
        ws();
        if (s[i] == ',') { ++i; continue; }
        if (s[i] == '}') { ++i; break; }
        fail("expected ',' or '}'");
      }
    } else if (c == '[') {
      j.kind = Json::Array;
      ++i;
      ws();
      if (s[i] == ']') { ++i; return j; }
      for (;;) {
        j.arr.push_back(value());
        ws();
        if (s[i] == ',') { ++i; continue; }
        if (s[i] == ']') { ++i; break; }
        fail("expected ',' or ']'");
      }
    } else if (c == '"') {
      j.kind = Json::String;
      j.str = str();
    } else if (lit("true")) {
      j.kind = Json::Bool; j.b = true;
    } else if (lit("false")) {
      j.kind = Json::Bool; j.b = false;
    } else if (lit("null")) {
      j.kind = Json::Null;
    } else {
      char* end = nullptr;
      j.num = std::strtod(s.c_str() + i, &end);
      if (end == s.c_str() + i) fail("unexpected character");
      i = size_t(end - s.c_str());
      j.kind = Json::Number;
    }
    return j;
  }
};

}  // namespace

Json parse_json(const std::string& text) {
  Parser p(text);
  Json j = p.value();
  p.ws();
  if (p.i != text.size()) p.fail("trailing characters");
  return j;
}

}  // namespace tdmix
