// cfs_scribble.cpp -- the scribble composition language (Section 3.1) lowered
// into the fused chain of the generated chaos-game program.
//
// Section 3.1 composes kernels from three kinds of fragments: verses
// (function-like code inlined at each call, with keyword arguments and their
// defaults), stanzas (like verses, with a split point where the caller's own
// block is injected) and poems (the top level that calls them).  Here a poem
// is the transform chain of one chaos-game step: its statements run on the
// copy of the point (qx, qy, qz), its colour index kc and the step's auxiliary
// random word aux, and splat into the render's targets.  Expansion rules:
//
//   __verse  NAME(p1, p2 | T k1 = d1; T k2 = d2;) { BODY }
//   __stanza NAME(p1 | T k = d;) { PRE __split_stanza(); POST }
//   __poem   NAME() { ... @VCALL v(a1, a2 | k1 = x;); ...
//                     @SCALL s(a1 | k = y;) { BLOCK } ... }
//
// A call becomes a block: each positional parameter is bound by reference to
// its argument expression (`auto&& p1 = (a1);`), each keyword parameter is a
// local of its declared type initialised with the call's value or else the
// default, then the body follows (for a stanza with the caller's expanded
// block in place of __split_stanza()).  Bodies may use the names of the
// calling context.  Calls expand recursively (depth <= 32).  Only the name of
// a positional declaration matters (its last identifier).
#include <cctype>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "cfs_internal.h"

namespace cfs {
namespace {

struct Fragment {
    bool stanza = false;
    std::vector<std::string> params;                          // positional names
    std::vector<std::pair<std::string, std::string>> kw;      // "T name" -> default
    std::vector<std::string> kw_names;
    std::string body;
};

bool is_ident(char c) { return std::isalnum((unsigned char)c) || c == '_'; }

// index just past the bracket that closes the one at `open` (skips string
// and character literals and comments); npos when unbalanced
size_t match_close(const std::string& s, size_t open)
{
    const char o = s[open];
    const char c = o == '(' ? ')' : (o == '{' ? '}' : ']');
    int depth = 0;
    for (size_t i = open; i < s.size(); ++i) {
        const char ch = s[i];
        if (ch == '"' || ch == '\'') {
            for (++i; i < s.size() && s[i] != ch; ++i)
                if (s[i] == '\\') ++i;
            continue;
        }
        if (ch == '/' && i + 1 < s.size() && s[i + 1] == '/') {
            while (i < s.size() && s[i] != '\n') ++i;
            continue;
        }
        if (ch == '/' && i + 1 < s.size() && s[i + 1] == '*') {
            const size_t e = s.find("*/", i + 2);
            if (e == std::string::npos) return std::string::npos;
            i = e + 1;
            continue;
        }
        if (ch == o) ++depth;
        else if (ch == c && --depth == 0) return i + 1;
    }
    return std::string::npos;
}

std::string trim(const std::string& s)
{
    size_t a = 0, b = s.size();
    while (a < b && std::isspace((unsigned char)s[a])) ++a;
    while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
    return s.substr(a, b - a);
}

// splits at `sep` outside brackets
std::vector<std::string> split_top(const std::string& s, char sep)
{
    std::vector<std::string> out;
    int depth = 0;
    size_t start = 0;
    for (size_t i = 0; i < s.size(); ++i) {
        const char ch = s[i];
        if (ch == '(' || ch == '[' || ch == '{') ++depth;
        else if (ch == ')' || ch == ']' || ch == '}') --depth;
        else if (ch == sep && depth == 0) {
            out.push_back(s.substr(start, i - start));
            start = i + 1;
        }
    }
    out.push_back(s.substr(start));
    return out;
}

std::string last_ident(const std::string& decl)
{
    size_t e = decl.size();
    while (e > 0 && !is_ident(decl[e - 1])) --e;
    size_t b = e;
    while (b > 0 && is_ident(decl[b - 1])) --b;
    return decl.substr(b, e - b);
}

bool parse_params(const std::string& inside, Fragment* f, std::string* err)
{
    const std::vector<std::string> halves = split_top(inside, '|');
    if (halves.size() > 2) { *err = "more than one '|' in a parameter list"; return false; }
    for (const std::string& p : split_top(halves[0], ',')) {
        const std::string t = trim(p);
        if (t.empty()) continue;
        const std::string n = last_ident(t);
        if (n.empty()) { *err = "positional parameter without a name: " + t; return false; }
        f->params.push_back(n);
    }
    if (halves.size() == 2) {
        for (const std::string& k : split_top(halves[1], ';')) {
            const std::string t = trim(k);
            if (t.empty()) continue;
            const size_t eq = t.find('=');
            if (eq == std::string::npos) { *err = "keyword parameter without a default: " + t; return false; }
            const std::string decl = trim(t.substr(0, eq));
            const std::string name = last_ident(decl);
            if (name.empty() || decl == name) {
                *err = "keyword parameter needs a type and a name: " + t;
                return false;
            }
            f->kw.push_back({decl, trim(t.substr(eq + 1))});
            f->kw_names.push_back(name);
        }
    }
    return true;
}

struct Program {
    std::map<std::string, Fragment> verses;   // verses and stanzas
    std::map<std::string, Fragment> poems;
};

bool parse_program(const std::string& src, Program* prog, std::string* err)
{
    static const char* kinds[] = {"__verse", "__stanza", "__poem"};
    size_t pos = 0;
    while (true) {
        size_t best = std::string::npos;
        int which = -1;
        for (int k = 0; k < 3; ++k) {
            size_t p = src.find(kinds[k], pos);
            while (p != std::string::npos &&
                   ((p > 0 && is_ident(src[p - 1])) ||
                    (p + std::strlen(kinds[k]) < src.size() &&
                     is_ident(src[p + std::strlen(kinds[k])]))))
                p = src.find(kinds[k], p + 1);
            if (p < best) { best = p; which = k; }
        }
        if (which < 0) break;
        size_t i = best + std::strlen(kinds[which]);
        while (i < src.size() && std::isspace((unsigned char)src[i])) ++i;
        const size_t n0 = i;
        while (i < src.size() && is_ident(src[i])) ++i;
        const std::string name = src.substr(n0, i - n0);
        while (i < src.size() && std::isspace((unsigned char)src[i])) ++i;
        if (name.empty() || i >= src.size() || src[i] != '(') {
            *err = std::string(kinds[which]) + " needs a name and a parameter list";
            return false;
        }
        const size_t pe = match_close(src, i);
        if (pe == std::string::npos) { *err = "unbalanced parameter list of " + name; return false; }
        Fragment f;
        f.stanza = which == 1;
        if (!parse_params(src.substr(i + 1, pe - i - 2), &f, err)) {
            *err = name + ": " + *err;
            return false;
        }
        size_t b = pe;
        while (b < src.size() && std::isspace((unsigned char)src[b])) ++b;
        if (b >= src.size() || src[b] != '{') { *err = name + ": missing body"; return false; }
        const size_t be = match_close(src, b);
        if (be == std::string::npos) { *err = name + ": unbalanced body"; return false; }
        f.body = src.substr(b + 1, be - b - 2);
        if (f.stanza && f.body.find("__split_stanza") == std::string::npos) {
            *err = "stanza " + name + " has no __split_stanza()";
            return false;
        }
        auto& table = which == 2 ? prog->poems : prog->verses;
        if (table.count(name) || (which == 2 ? prog->verses.count(name) : prog->poems.count(name))) {
            *err = "duplicate name " + name;
            return false;
        }
        table[name] = f;
        pos = be;
    }
    return true;
}

bool expand(const Program& prog, const std::string& text, int depth, std::string* out,
            std::string* err);

// one @VCALL / @SCALL expansion; `block` is the caller's block of an @SCALL
bool expand_call(const Program& prog, const std::string& name, const std::string& inside,
                 bool scall, const std::string& block, int depth, std::string* out,
                 std::string* err)
{
    auto it = prog.verses.find(name);
    if (it == prog.verses.end()) { *err = "unknown verse or stanza " + name; return false; }
    const Fragment& f = it->second;
    if (f.stanza != scall) {
        *err = name + (scall ? " is a verse: call it with @VCALL" : " is a stanza: call it with @SCALL");
        return false;
    }
    Fragment call;
    {
        // the call's own list: positional arguments, then `name = value;` overrides
        const std::vector<std::string> halves = split_top(inside, '|');
        if (halves.size() > 2) { *err = name + ": more than one '|' in a call"; return false; }
        std::vector<std::string> args;
        for (const std::string& a : split_top(halves[0], ',')) {
            const std::string t = trim(a);
            if (!t.empty()) args.push_back(t);
        }
        if (args.size() != f.params.size()) {
            std::ostringstream m;
            m << name << ": " << args.size() << " positional arguments for " << f.params.size()
              << " parameters";
            *err = m.str();
            return false;
        }
        std::map<std::string, std::string> over;
        if (halves.size() == 2) {
            for (const std::string& k : split_top(halves[1], ';')) {
                const std::string t = trim(k);
                if (t.empty()) continue;
                const size_t eq = t.find('=');
                if (eq == std::string::npos) { *err = name + ": keyword without a value: " + t; return false; }
                const std::string kn = trim(t.substr(0, eq));
                bool known = false;
                for (const auto& n : f.kw_names) known = known || n == kn;
                if (!known) { *err = name + ": no keyword parameter " + kn; return false; }
                over[kn] = trim(t.substr(eq + 1));
            }
        }
        std::ostringstream s;
        s << "{ /* " << (scall ? "stanza " : "verse ") << name << " */\n";
        for (size_t j = 0; j < args.size(); ++j)
            s << "auto&& " << f.params[j] << " = (" << args[j] << ");\n";
        for (size_t j = 0; j < f.kw.size(); ++j) {
            const std::string& n = f.kw_names[j];
            const std::string v = over.count(n) ? over[n] : f.kw[j].second;
            s << f.kw[j].first << " = (" << v << ");\n";
        }
        for (size_t j = 0; j < f.params.size(); ++j) s << "(void)" << f.params[j] << ";\n";
        for (const auto& n : f.kw_names) s << "(void)" << n << ";\n";
        std::string body = f.body;
        if (scall) {
            const size_t sp = body.find("__split_stanza");
            const size_t open = body.find('(', sp);
            size_t close = open == std::string::npos ? std::string::npos : match_close(body, open);
            if (close == std::string::npos) { *err = name + ": malformed __split_stanza()"; return false; }
            while (close < body.size() && std::isspace((unsigned char)body[close])) ++close;
            if (close < body.size() && body[close] == ';') ++close;
            body = body.substr(0, sp) + "{\n" + block + "\n}\n" + body.substr(close);
        }
        std::string expanded;
        if (!expand(prog, body, depth + 1, &expanded, err)) return false;
        s << expanded << "\n}\n";
        *out += s.str();
    }
    return true;
}

bool expand(const Program& prog, const std::string& text, int depth, std::string* out,
            std::string* err)
{
    if (depth > 32) { *err = "calls nested deeper than 32 (recursion?)"; return false; }
    size_t pos = 0;
    while (true) {
        const size_t at = text.find('@', pos);
        if (at == std::string::npos) { *out += text.substr(pos); return true; }
        *out += text.substr(pos, at - pos);
        const bool v = text.compare(at, 6, "@VCALL") == 0;
        const bool sc = text.compare(at, 6, "@SCALL") == 0;
        if (!v && !sc) { *err = "unknown directive at '" + text.substr(at, 12) + "'"; return false; }
        size_t i = at + 6;
        while (i < text.size() && std::isspace((unsigned char)text[i])) ++i;
        const size_t n0 = i;
        while (i < text.size() && is_ident(text[i])) ++i;
        const std::string name = text.substr(n0, i - n0);
        while (i < text.size() && std::isspace((unsigned char)text[i])) ++i;
        if (name.empty() || i >= text.size() || text[i] != '(') {
            *err = "a call needs a name and an argument list";
            return false;
        }
        const size_t pe = match_close(text, i);
        if (pe == std::string::npos) { *err = name + ": unbalanced argument list"; return false; }
        const std::string inside = text.substr(i + 1, pe - i - 2);
        size_t next = pe;
        std::string block;
        if (sc) {
            size_t b = pe;
            while (b < text.size() && std::isspace((unsigned char)text[b])) ++b;
            if (b >= text.size() || text[b] != '{') { *err = name + ": @SCALL needs a block"; return false; }
            const size_t be = match_close(text, b);
            if (be == std::string::npos) { *err = name + ": unbalanced block"; return false; }
            std::string inner;
            if (!expand(prog, text.substr(b + 1, be - b - 2), depth + 1, &inner, err)) return false;
            block = inner;
            next = be;
        } else {
            while (next < text.size() && std::isspace((unsigned char)text[next])) ++next;
            if (next < text.size() && text[next] == ';') ++next;
        }
        if (!expand_call(prog, name, inside, sc, block, depth, out, err)) return false;
        pos = next;
    }
}

}  // namespace

cfs_status scribble_expand(const std::string& source, const std::string& poem, std::string* body,
                           std::vector<int>* splat_slots)
{
    Program prog;
    std::string err;
    if (!parse_program(source, &prog, &err)) return fail(CFS_ERR_INVALID_ARG, "scribble: " + err);
    auto it = prog.poems.find(poem);
    if (it == prog.poems.end()) return fail(CFS_ERR_INVALID_ARG, "scribble: no poem " + poem);
    if (!it->second.params.empty() || !it->second.kw.empty())
        return fail(CFS_ERR_INVALID_ARG, "scribble: a chain poem takes no parameters (it works "
                                         "on qx, qy, qz, kc, aux, px, py, pz, k)");
    std::string out;
    if (!expand(prog, it->second.body, 0, &out, &err))
        return fail(CFS_ERR_INVALID_ARG, "scribble: " + err);
    // splat(N) calls: each gets a static record index; the slots must be
    // integer literals (the target kind is compiled in)
    splat_slots->clear();
    std::string res;
    size_t pos = 0;
    while (true) {
        size_t p = out.find("splat", pos);
        while (p != std::string::npos &&
               ((p > 0 && is_ident(out[p - 1])) || (p + 5 < out.size() && is_ident(out[p + 5]))))
            p = out.find("splat", p + 1);
        if (p == std::string::npos) { res += out.substr(pos); break; }
        size_t i = p + 5;
        while (i < out.size() && std::isspace((unsigned char)out[i])) ++i;
        if (i >= out.size() || out[i] != '(') { res += out.substr(pos, i - pos); pos = i; continue; }
        const size_t pe = match_close(out, i);
        if (pe == std::string::npos) return fail(CFS_ERR_INVALID_ARG, "scribble: unbalanced splat(");
        const std::string a = trim(out.substr(i + 1, pe - i - 2));
        if (a.size() != 1 || a[0] < '0' || a[0] >= '0' + CFS_MAX_TARGETS)
            return fail(CFS_ERR_INVALID_ARG, "scribble: splat(slot) needs a literal slot 0..3");
        std::ostringstream m;
        m << "CFS_SCRIBBLE_SPLAT_" << splat_slots->size() << "()";
        res += out.substr(pos, p - pos) + m.str();
        splat_slots->push_back(a[0] - '0');
        pos = pe;
    }
    if (splat_slots->size() > 32)
        return fail(CFS_ERR_INVALID_ARG, "scribble: at most 32 splat calls");
    *body = res;
    return CFS_OK;
}

}  // namespace cfs
