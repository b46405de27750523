#include "netdesc.h"

#include <map>
#include <set>
#include <sstream>

namespace nvisr {

int NetDesc::find(const std::string &name) const {
    for (size_t i = 0; i < layers.size(); ++i)
        if (layers[i].name == name) return (int)i;
    return -1;
}

static std::vector<std::string> split(const std::string &s, char sep) {
    std::vector<std::string> out;
    std::string cur;
    for (char c : s) {
        if (c == sep) {
            out.push_back(cur);
            cur.clear();
        } else {
            cur += c;
        }
    }
    out.push_back(cur);
    return out;
}

static bool to_int(const std::string &s, int *v) {
    if (s.empty()) return false;
    char *end = nullptr;
    long x = strtol(s.c_str(), &end, 10);
    if (*end) return false;
    *v = (int)x;
    return true;
}

bool parse_netdesc(const char *text, int64_t blob_count, NetDesc *net, std::string *err) {
    if (!text) {
        *err = "network description is NULL";
        return false;
    }
    std::istringstream in(text);
    std::string line;
    bool header = false;
    int lineno = 0;
    int64_t pos = 0;
    std::set<std::string> known;  // tensors defined so far
    auto fail = [&](const std::string &m) {
        *err = "line " + std::to_string(lineno) + ": " + m;
        return false;
    };
    while (std::getline(in, line)) {
        ++lineno;
        const size_t hash = line.find('#');
        if (hash != std::string::npos) line = line.substr(0, hash);
        std::istringstream ls(line);
        std::vector<std::string> tok;
        for (std::string t; ls >> t;) tok.push_back(t);
        if (tok.empty()) continue;
        if (!header) {
            if (tok.size() != 2 || tok[0] != "nvisr-net" || tok[1] != "1") return fail("expected 'nvisr-net 1'");
            header = true;
            continue;
        }
        const std::string &key = tok[0];
        if (key == "family") {
            if (tok.size() != 2 || (tok[1] != "tuple" && tok[1] != "group")) return fail("bad family");
            net->family = tok[1];
        } else if (key == "scale") {
            // horizontal and vertical scale (Section 3.2), or one for both
            int sx, sy;
            if (tok.size() < 2 || tok.size() > 3 || !to_int(tok[1], &sx) || sx < 1 || sx > 16) return fail("bad scale");
            sy = sx;
            if (tok.size() == 3 && (!to_int(tok[2], &sy) || sy < 1 || sy > 16)) return fail("bad scale");
            net->scale = sx;
            net->scale_y = sy;
        } else if (key == "frames" || key == "align") {
            int v;
            if (tok.size() != 2 || !to_int(tok[1], &v) || v < 1 || v > 16) return fail("bad " + key);
            (key == "frames" ? net->frames : net->align) = v;
        } else if (key == "flags") {
            if (tok.size() != 2) return fail("bad flags");
            for (const std::string &f : split(tok[1], ',')) {
                if (f == "interp") net->interp = true;
                else if (f == "extra") net->extra = true;
                else if (f == "double") net->dbl = true;
                else return fail("unknown flag " + f);
            }
        } else if (key == "domain") {
            if (tok.size() != 2 || (tok[1] != "rgb" && tok[1] != "yuv")) return fail("bad domain (rgb or yuv)");
            net->yuv = tok[1] == "yuv";
        } else if (key == "skip") {
            if (tok.size() != 2) return fail("bad skip");
            if (tok[1] == "none") net->skip = 0;
            else if (tok[1] == "nearest") net->skip = 1;
            else if (tok[1] == "bilinear") net->skip = 2;
            else return fail("unknown skip " + tok[1]);
        } else if (key == "conv" || key == "dcn") {
            if (tok.size() < 2) return fail("layer without name");
            NetLayer L;
            L.op = key;
            L.name = tok[1];
            std::map<std::string, std::string> kv;
            for (size_t i = 2; i < tok.size(); ++i) {
                const size_t eq = tok[i].find('=');
                if (eq == std::string::npos) return fail("expected key=value, got " + tok[i]);
                kv[tok[i].substr(0, eq)] = tok[i].substr(eq + 1);
            }
            if (!kv.count("in") || !kv.count("cin") || !kv.count("cout")) return fail("layer needs in, cin, cout");
            L.in = split(kv["in"], ',');
            if (!to_int(kv["cin"], &L.cin) || !to_int(kv["cout"], &L.cout) || L.cin < 1 || L.cout < 1 ||
                L.cin > 1024 || L.cout > 1024)
                return fail("bad cin/cout");
            if (key == "conv") {
                if (!kv.count("k") || !to_int(kv["k"], &L.k) || (L.k != 1 && L.k != 3)) return fail("k must be 1 or 3");
                const std::string act = kv.count("act") ? kv["act"] : "none";
                if (act == "lrelu") L.act = 1;
                else if (act != "none") return fail("unknown act " + act);
            } else {
                L.k = 3;
                if (!kv.count("om") || !kv.count("groups") || !to_int(kv["groups"], &L.groups) || L.groups < 1 ||
                    L.cin % L.groups)
                    return fail("dcn needs om and groups dividing cin");
                L.om = kv["om"];
                if (!known.count(L.om)) return fail("unknown om source " + L.om);
            }
            if (kv.count("ps") && (kv.count("psx") || kv.count("psy"))) return fail("ps with psx/psy");
            if (kv.count("ps")) {
                if (!to_int(kv["ps"], &L.ps) || L.ps != 2 || L.cout % 4) return fail("ps must be 2 with cout divisible by 4");
                L.psy = L.psx = 2;
            } else if (kv.count("psx") || kv.count("psy")) {
                if ((kv.count("psx") && (!to_int(kv["psx"], &L.psx) || L.psx < 1 || L.psx > 2)) ||
                    (kv.count("psy") && (!to_int(kv["psy"], &L.psy) || L.psy < 1 || L.psy > 2)))
                    return fail("psx / psy must be 1 or 2");
                if (L.cout % (L.psx * L.psy)) return fail("cout must be divisible by psx * psy");
                if (L.psx == 2 && L.psy == 2) L.ps = 2;  // the same as ps=2
            }
            if (kv.count("add")) {
                L.add = kv["add"];
                if (!known.count(L.add)) return fail("unknown add source " + L.add);
            }
            for (const std::string &s : L.in)
                if (!known.count(s) && s != "tuple" && s.rfind("frame", 0) != 0) return fail("unknown source " + s);
            if (kv.count("share")) {
                L.share = kv["share"];
                const int o = net->find(L.share);
                if (o < 0) return fail("unknown share " + L.share);
                const NetLayer &S = net->layers[o];
                if (S.cin != L.cin || S.cout != L.cout || S.k != L.k || S.op != L.op) return fail("share shape mismatch");
                L.owner = S.owner;
                L.woff = S.woff;
            } else {
                L.owner = (int)net->layers.size();
                L.woff = pos;
                pos += (int64_t)L.cout * L.cin * L.k * L.k + L.cout;
            }
            known.insert(L.name);
            net->layers.push_back(L);
        } else if (key == "pool" || key == "up") {
            // weightless resampling of the extract stage's pyramid (Section 3.1): a 2x2 mean,
            // or a bilinear x2 upsample; cin = cout = the source's channels
            if (tok.size() != 4) return fail(key + " needs a name, in= and cin=");
            NetLayer L;
            L.op = key;
            L.name = tok[1];
            L.k = 1;
            for (size_t i = 2; i < 4; ++i) {
                if (tok[i].rfind("in=", 0) == 0) L.in = {tok[i].substr(3)};
                else if (tok[i].rfind("cin=", 0) == 0 && to_int(tok[i].substr(4), &L.cin)) L.cout = L.cin;
                else return fail("bad " + key + " attribute " + tok[i]);
            }
            if (L.in.size() != 1 || L.cin < 1 || L.cin > 1024) return fail(key + " needs in= and cin=");
            if (!known.count(L.in[0])) return fail("unknown source " + L.in[0]);
            L.owner = (int)net->layers.size();
            known.insert(L.name);
            net->layers.push_back(L);
        } else if (key == "out") {
            if (tok.size() < 2) return fail("out without name");
            NetOutput o;
            o.name = tok[1];
            if (net->find(o.name) < 0) return fail("unknown output " + o.name);
            for (size_t i = 2; i < tok.size(); ++i) {
                if (tok[i].rfind("skip=", 0) != 0) return fail("unknown out attribute " + tok[i]);
                o.skip = split(tok[i].substr(5), ',');
            }
            net->outputs.push_back(o);
        } else {
            return fail("unknown statement " + key);
        }
    }
    if (!header) {
        *err = "empty network description";
        return false;
    }
    if (net->layers.empty() || net->outputs.empty()) {
        *err = "network has no layers or no outputs";
        return false;
    }
    if (pos != blob_count) {
        *err = "weight blob has " + std::to_string(blob_count) + " floats, description uses " + std::to_string(pos);
        return false;
    }
    net->weights_used = pos;
    return true;
}

}  // namespace nvisr
