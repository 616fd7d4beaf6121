#include "qss_driver.h"

#include <dlfcn.h>

#include <mutex>

#define QSS_STR(x) #x
#define QSS_XSTR(x) QSS_STR(x)

namespace qss {
Driver& drv() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_GLOBAL);
    if (!h) return;
    bool all = true;
#define QSS_DRV_LOAD(f)                                      \
    d.f = (decltype(d.f))dlsym(h, QSS_XSTR(f));               \
    if (!d.f) all = false;
    QSS_DRV_FUNCS(QSS_DRV_LOAD)
#undef QSS_DRV_LOAD
    d.ok = all;
  });
  return d;
}
}  // namespace qss
